"""Helpers shared by the GPU parity tests (oracle on the CPU, CUDA path through the C ABI)."""
import numpy as np

import oracle


def oracle_blocks(P, V):
    """The oracle's divergence (and viscous) rows in the library's per-vertex block layout:
    for each active vertex, rows d_0, d_x, d_y over the data in ascending column order
    (f_1, g_1, ..., f_N, g_N by vertex id, then edge fluxes by edge index)."""
    blocks = []
    D = [d.tocsr() for d in P.D]
    for d in D:
        d.sort_indices()
    for r in range(len(P.active)):
        blocks.append(np.concatenate([d.data[d.indptr[r]:d.indptr[r + 1]] for d in D]))
    out = {"div_coef": np.concatenate(blocks)}
    if getattr(P, "Dv", None) is not None:
        Dv = [d.tocsr() for d in P.Dv]
        for d in Dv:
            d.sort_indices()
        out["visc_coef"] = np.concatenate(
            [np.concatenate([d.data[d.indptr[r]:d.indptr[r + 1]] for d in Dv])
             for r in range(len(P.active))])
    return out


def inject_oracle_coefficients(prep, P, V):
    """Overwrite the library's geometry coefficients with the oracle's, after checking that
    both sides agree on every discrete choice (stencils, flux-edge set, CSR structure)."""
    assert np.array_equal(prep.get("flux_edges"), P.edges)
    assert np.array_equal(prep.get("stencil").reshape(-1, 6), P.stencil)
    assert np.array_equal(prep.get("active"), P.active)
    prep.set("w5", P.w5.ravel())
    prep.set("w3", P.w3.ravel())
    for k, v in oracle_blocks(P, V).items():
        assert len(v) == len(prep.get(k)), k
        prep.set(k, v)


def oracle_with_library_coefficients(P, prep):
    """The oracle's preprocessing with the library's own geometry coefficients put in (5-node
    and 3-node weights, divergence and viscous rows), after checking that both sides made the
    same discrete choices.  The oracle's residual on it is the method's arithmetic on exactly
    the coefficients the library's full path uses."""
    import copy
    assert np.array_equal(prep.get("flux_edges"), P.edges)
    assert np.array_equal(prep.get("stencil").reshape(-1, 6), P.stencil)
    assert np.array_equal(prep.get("active"), P.active)
    Q = copy.copy(P)
    Q.w5 = prep.get("w5").reshape(P.w5.shape).copy()
    Q.w3 = prep.get("w3").reshape(P.w3.shape).copy()

    def put(mats, flat):
        out = []
        off = 0
        n = len(P.active)
        ms = [d.tocsr().copy() for d in mats]
        for d in ms:
            d.sort_indices()
        for r in range(n):
            for d in ms:
                a, b = d.indptr[r], d.indptr[r + 1]
                d.data[a:b] = flat[off:off + (b - a)]
                off += b - a
        assert off == len(flat)
        return ms
    Q.D = put(P.D, prep.get("div_coef"))
    if getattr(P, "Dv", None) is not None:
        Q.Dv = put(P.Dv, prep.get("visc_coef"))
    return Q


def elementwise_rel(R, R_ref, cols=None):
    """Largest |R - R_ref| / (|R_ref| + rms of R_ref over the entry's row group) over every
    entry: an element-wise bound with a floor, so that no single vertex can hide under a norm,
    while entries near a zero of the residual are measured against their group's scale."""
    if cols is not None:
        R, R_ref = R[:, cols], R_ref[:, cols]
    worst = 0.0
    for g in range(3):
        a, b = R[4 * g:4 * g + 4], R_ref[4 * g:4 * g + 4]
        floor = np.sqrt(np.mean(b * b))
        worst = max(worst, float(np.max(np.abs(a - b) / (np.abs(b) + floor))))
    return worst


def rel_l2_groups(R, R_ref, cols=None):
    """Relative L2 error of the w, w_x and w_y row groups (rows 0-3, 4-7, 8-11)."""
    if cols is not None:
        R, R_ref = R[:, cols], R_ref[:, cols]
    out = []
    for g in range(3):
        a, b = R[4 * g:4 * g + 4], R_ref[4 * g:4 * g + 4]
        out.append(float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)))
    return out


def near_threshold_vertices(m, P, U, opts, margin=1e-9):
    """Active vertices whose divergence reads an edge whose WENO sensor value lies within
    `margin` of a threshold: there the branch is decided by rounding, and either side is a
    correct evaluation of the method."""
    diag = {}
    oracle.hfd_oracle.edge_values(P, U.copy(), opts, diag)
    o1 = np.stack(diag["omega1"])            # (2, Ee, 4)
    d = np.minimum(np.abs(o1 - opts.sens_lo), np.abs(o1 - opts.sens_hi)).min(axis=(0, 2))
    bad_edges = set(P.edges[d < margin].tolist())
    if not bad_edges:
        return np.zeros(0, dtype=np.int64)
    V = len(m["x"])
    D = P.D[0].tocsr()
    bad = []
    for r in range(len(P.active)):
        cols = D.indices[D.indptr[r]:D.indptr[r + 1]]
        e = cols[cols >= 2 * V] - 2 * V
        if bad_edges.intersection(e.tolist()):
            bad.append(P.active[r])
    return np.array(bad, dtype=np.int64)


def checked_build_cases():
    """Small meshes covering every gather of the forward kernels (periodic, transmissive ghosts,
    fixed wall bands, viscous rows, a Delaunay mesh, FP32 chunks, the persistent launch):
    name -> (mesh, state, Mesh keywords, persistent launch)."""
    import synth
    v = synth.jittered_grid(24, 24, 10.0, 10.0, seed=1)
    q = synth.jittered_box_with_ghosts(24, 24, (0.0, 1.0), (0.0, 1.0), 5, seed=2)
    t = synth.jittered_grid(16, 16, 2 * np.pi, 2 * np.pi, seed=3)
    c = synth.couette_channel(16, 17, 6, seed=7)
    s = synth.embedded_circle_box(16, seed=8)
    visc_t = dict(viscous=True, mu=0.01, prandtl=0.72, R_gas=1.0 / (1.4 * 0.01))
    visc_c = dict(viscous=True, mu=0.1, prandtl=100.0, R_gas=0.4 * 10.0 / 1.4)
    return {
        "vortex_fp64": (v, synth.isentropic_vortex(v), {}, False),
        "vortex_fp32": (v, synth.isentropic_vortex(v), {"precision": "fp32"}, False),
        "vortex_persistent": (v, synth.isentropic_vortex(v), {}, True),
        "quad_fp64": (q, synth.four_quadrant(q), {}, False),
        "quad_fp32": (q, synth.four_quadrant(q), {"precision": "fp32"}, False),
        "tgv_viscous": (t, synth.taylor_green(t), visc_t, False),
        "couette_walls": (c, synth.couette(c), visc_c, False),
        "circular_sod": (s, synth.circular_sod(s), {}, False),
    }


def run_checked_build_cases(pkg, torch):
    """Residual and two device-CFL steps of every case; raises if a mesh's error word is set."""
    out = {}
    for name, (m, U, kw, persistent) in checked_build_cases().items():
        mesh = pkg.Mesh(m, **kw)
        if persistent:
            mesh.set_launch(True, 0)
        X = mesh.import_state(torch.from_numpy(U).cuda())
        out[name + "/R"] = mesh.export_state(mesh.residual(X)).cpu().numpy()
        mesh.steps(X, 0.0, 2)
        out[name + "/U"] = mesh.export_state(X).cpu().numpy()
        mesh.check()
    return out


def c2_chunk_oracle_residual(task):
    """Spawned worker: the oracle's residual of the n x n four-quadrant mesh (5 ghost layers)
    at a chunk of active vertices, on the library's own coefficients for that chunk (loaded
    from the .npz of its preprocessing arrays), and the chunk's vertices that read an edge
    whose sensor lies within 1e-9 of a threshold.  The discrete structure -- every needed
    edge's 6-node stencil (Sec. 2.1) and each vertex's two-level set (R7) -- comes from the
    oracle's own functions and must equal the library's; the coefficient solves are not
    repeated (the coefficients are the library's, compared elsewhere).  Returns (chunk,
    R[:, chunk], near-threshold vertices)."""
    import scipy.sparse as sp
    import synth
    from oracle import hfd_oracle as H
    n, chunk, lib_path = task
    with np.load(lib_path) as z:                # every array read once
        lib = {k: z[k] for k in z.files}
    m = synth.jittered_box_with_ghosts(n, n, (0.0, 1.0), (0.0, 1.0), 5, seed=2)
    U = synth.four_quadrant(m)
    topo = oracle.build_topology(m)
    V, E = topo["V"], len(topo["edges"])
    sets = [oracle.vertex_stencil(topo, int(v)) for v in chunk]
    need = np.array(sorted(set(int(e) for _, es in sets for e in es)), dtype=np.int64)
    P = H.Prep()
    P.topo, P.active, P.opts, P.edges = topo, np.asarray(chunk, dtype=np.int64), oracle.Options(), need
    geo = [oracle.edge_geometry(m, topo, int(e)) for e in need]
    P.stencil = np.array([g[0] for g in geo], dtype=np.int64).reshape(-1, 6)
    P.normal = np.array([g[3] for g in geo]).reshape(-1, 2)
    fe = lib["flux_edges"]
    pos = np.searchsorted(fe, need)
    assert np.array_equal(fe[pos], need)
    assert np.array_equal(lib["stencil"].reshape(-1, 6)[pos], P.stencil)
    P.w5 = lib["w5"].reshape(-1, 2, 15)[pos].copy()
    P.w3 = lib["w3"].reshape(-1, 2, 3, 3)[pos].copy()
    act = lib["active"]
    rl = np.searchsorted(act, chunk)
    assert np.array_equal(act[rl], chunk)
    N = np.diff(lib["div_vptr"])
    M = np.diff(lib["div_eptr"])
    off = np.concatenate([[0], np.cumsum(3 * (2 * N + M))])
    cols, vals, ptr = [], [[], [], []], [0]
    for (verts, edges), r in zip(sets, rl):
        assert len(verts) == N[r] and len(edges) == M[r]
        c = np.concatenate([np.stack([2 * verts, 2 * verts + 1], 1).ravel(), 2 * V + edges])
        L = len(c)
        blk = lib["div_coef"][off[r]:off[r] + 3 * L]
        cols.append(c)
        for k in range(3):
            vals[k].append(blk[k * L:(k + 1) * L])
        ptr.append(ptr[-1] + L)
    cols = np.concatenate(cols)
    P.D = [sp.csr_matrix((np.concatenate(vals[k]), cols, np.array(ptr)), shape=(len(chunk), 2 * V + E))
           for k in range(3)]
    R = oracle.residual(m, P, U.copy())
    bad = near_threshold_vertices(m, P, U, P.opts)
    return chunk, R[:, chunk], bad
