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
