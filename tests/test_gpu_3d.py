"""GPU parity of the three-dimensional extension (include/hfd3d.h) against its FP64 oracle
(oracle/hfd3d.py): the preprocessing's discrete choices and coefficients, the residual with the
oracle's coefficients injected (kernel parity: smooth, shock and forced-branch data), three
SSP-RK3 steps, the library's own coefficients end to end, and the error word."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import hfd3d as O          # noqa: E402
from synth import three_d as T         # noqa: E402

N = 8                                  # 8^3 vertices: 3584 edges, ~500 entries per row


def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2109_01286_gb300 import hfd3d
    return hfd3d


@pytest.fixture(scope="module")
def box():
    m = T.periodic_tet_box(N, N, N, 10.0, 10.0, 10.0, seed=3)
    P = O.prepare(m)
    return m, P


def _groups(R, R_ref):
    """Relative L2 error of the row groups w, w_x, w_y, w_z (rows 0-4, 5-9, 10-14, 15-19)."""
    return [float(np.linalg.norm(R[5 * g:5 * g + 5] - R_ref[5 * g:5 * g + 5]) /
                  max(np.linalg.norm(R_ref[5 * g:5 * g + 5]), 1e-300)) for g in range(4)]


def _elementwise(R, R_ref):
    """Largest |R - R_ref| / (|R_ref| + rms of the entry's row group)."""
    worst = 0.0
    for g in range(4):
        a, b = R[5 * g:5 * g + 5], R_ref[5 * g:5 * g + 5]
        floor = np.sqrt(np.mean(b * b))
        worst = max(worst, float(np.max(np.abs(a - b) / (np.abs(b) + floor))))
    return worst


def _inject(mesh, P):
    """Overwrite the device mesh's stencils, frames, weights and divergence coefficients with
    the oracle's (the connectivity must already agree)."""
    V = P.topo["V"]
    mesh.prep_set("sten", P.stencil.astype(np.int32))
    mesh.prep_set("frame", np.concatenate([P.normal, P.t1, P.t2], 1))
    mesh.prep_set("w5", P.w5)
    mesh.prep_set("w3", P.w3)
    vptr, vidx = mesh.prep_get("vptr"), mesh.prep_get("vidx")
    eptr, eidx = mesh.prep_get("eptr"), mesh.prep_get("eidx")
    cv = np.zeros((len(vidx), 4, 3))
    ce = np.zeros((len(eidx), 4))
    D = [P.D[r].tocsr() for r in range(4)]
    for v in range(V):
        for r in range(4):
            row = D[r].getrow(v)
            lut = dict(zip(row.indices.tolist(), row.data.tolist()))
            for j in range(vptr[v], vptr[v + 1]):
                u = int(vidx[j])
                for f in range(3):
                    cv[j, r, f] = lut.get(3 * u + f, 0.0)
            for j in range(eptr[v], eptr[v + 1]):
                ce[j, r] = lut.get(3 * V + int(eidx[j]), 0.0)
    mesh.prep_set("cv", cv)
    mesh.prep_set("ce", ce)


def _residual(mesh, U):
    Ud = torch.from_numpy(np.ascontiguousarray(U)).cuda()
    R = mesh.residual(Ud)
    torch.cuda.synchronize()
    mesh.check()
    return R.cpu().numpy()


def test_3d_structure_and_coefficients_match_the_oracle(box):
    """Discrete choices (edges, stencils, two-level sets, ranks) equal the oracle's; frames and
    3-node weights to rounding; 5-node weights and divergence rows within what the conditioning
    of their systems allows (sigma_min / sigma_max of the 20 x 20 Hermite systems reaches 1e-11,
    so LAPACK's and the Jacobi SVD's rows differ by rounding amplified that much)."""
    h = _cuda()
    m, P = box
    mesh = h.Mesh3(m)
    topo = P.topo
    assert np.array_equal(mesh.prep_get("edges").reshape(-1, 2), topo["edges"])
    assert np.array_equal(mesh.prep_get("sten").reshape(-1, 6), P.stencil)
    assert np.array_equal(mesh.prep_get("rank").reshape(-1, 2), P.rank)
    frame = mesh.prep_get("frame").reshape(-1, 9)
    np.testing.assert_allclose(frame, np.concatenate([P.normal, P.t1, P.t2], 1), atol=1e-15)
    np.testing.assert_allclose(mesh.prep_get("w3").reshape(P.w3.shape), P.w3, rtol=1e-12, atol=1e-14)
    w5 = mesh.prep_get("w5").reshape(P.w5.shape)
    assert np.abs(w5 - P.w5).max() < 1e-4
    assert np.median(np.abs(w5 - P.w5).max(axis=(1, 2))) < 1e-9
    vptr, vidx = mesh.prep_get("vptr"), mesh.prep_get("vidx")
    for v in range(0, topo["V"], 37):
        verts, edges = O.vertex_stencil(topo, v)
        assert np.array_equal(vidx[vptr[v]:vptr[v + 1]], verts)
    info = mesh.info()
    assert info["nv"] == N ** 3 and info["nedges"] == len(topo["edges"])
    assert info["rank_deficient_sides"] == int((P.rank < 20).sum())


@pytest.mark.parametrize("state", ["vortex", "wave", "sod"])
def test_3d_kernel_parity_residual(box, state):
    """With the oracle's coefficients injected, the residual matches the oracle to 1e-12 in L2
    per row group and 1e-10 element-wise, on smooth data (vortex tube, density wave) and on Sod
    data, where the sensor selects the weighted 3-node values near the two discontinuities."""
    h = _cuda()
    m, P = box
    U = {"vortex": lambda: T.vortex_tube(m),
         "wave": lambda: T.density_wave(m, amp=0.1),
         "sod": lambda: T.planar_sod3(m)}[state]()
    mesh = h.Mesh3(m)
    _inject(mesh, P)
    R = _residual(mesh, U)
    Rref = O.residual(m, P, U)
    assert max(_groups(R, Rref)) < 1e-12
    assert _elementwise(R, Rref) < 1e-10


@pytest.mark.parametrize("branch", ["hermite", "weno"])
def test_3d_kernel_parity_forced_branches(box, branch):
    """Every side forced to the 5-node or to the weighted 3-node value (testing aid), on the
    vortex tube: the two branches of Alg. 1 each match the oracle with nothing excluded."""
    h = _cuda()
    m, P = box
    U = T.vortex_tube(m)
    mesh = h.Mesh3(m, force_branch=branch)
    _inject(mesh, P)
    R = _residual(mesh, U)
    Rref = O.residual(m, P, U, O.Options3(force_branch=branch))
    assert max(_groups(R, Rref)) < 1e-12
    assert _elementwise(R, Rref) < 1e-10


def test_3d_steps_parity(box):
    """Three SSP-RK3 steps of fixed size (the oracle's CFL step of the initial state) on the
    vortex tube, with the oracle's coefficients: the states agree to 1e-11 relative."""
    h = _cuda()
    m, P = box
    U = T.vortex_tube(m)
    dt = O.cfl_dt(m, P, U)
    mesh = h.Mesh3(m)
    _inject(mesh, P)
    X = torch.from_numpy(U.copy()).cuda()
    mesh.steps(X, dt, 3)
    torch.cuda.synchronize()
    mesh.check()
    ref = U.copy()
    for _ in range(3):
        ref = O.step(m, P, ref, dt)
    X = X.cpu().numpy()
    assert max(_groups(X - U, ref - U)) < 1e-11
    assert float(np.abs(X - ref).max() / np.abs(ref).max()) < 1e-13


def test_3d_library_coefficients_end_to_end(box):
    """The library's own preprocessing end to end against the oracle: the residuals differ only
    by what the coefficient differences allow (the 5-node weights of ill-conditioned stencils),
    measured against the same residual evaluated by the oracle with the library's coefficients
    (which must then match to 1e-12)."""
    h = _cuda()
    m, P = box
    U = T.vortex_tube(m)
    mesh = h.Mesh3(m)
    R = _residual(mesh, U)
    Rref = O.residual(m, P, U)
    assert max(_groups(R, Rref)) < 1e-6
    # the oracle's arithmetic on the library's weights and rows
    import copy
    P2 = copy.copy(P)
    P2.w5 = mesh.prep_get("w5").reshape(P.w5.shape)
    P2.w3 = mesh.prep_get("w3").reshape(P.w3.shape)
    V = P.topo["V"]
    vptr, vidx = mesh.prep_get("vptr"), mesh.prep_get("vidx")
    eptr, eidx = mesh.prep_get("eptr"), mesh.prep_get("eidx")
    cv, ce = mesh.prep_get("cv").reshape(-1, 4, 3), mesh.prep_get("ce").reshape(-1, 4)
    import scipy.sparse as sp
    rows = np.concatenate([np.repeat(np.arange(V), np.diff(vptr) * 3),
                           np.repeat(np.arange(V), np.diff(eptr))])
    cols = np.concatenate([(3 * vidx[:, None] + np.arange(3)[None]).ravel(), 3 * V + eidx])
    P2.D = [sp.csr_matrix((np.concatenate([cv[:, r, :].ravel(), ce[:, r]]), (rows, cols)),
                          shape=(V, 3 * V + len(P.topo["edges"]))) for r in range(4)]
    R2 = O.residual(m, P2, U)
    assert max(_groups(R, R2)) < 1e-12


def test_3d_freestream_and_error_word(box):
    h = _cuda()
    m, P = box
    mesh = h.Mesh3(m)
    U = T.uniform_state3(m)
    R = _residual(mesh, U)
    assert np.abs(R).max() < 1e-11
    # a negative density makes the Roe averages non-finite: the error word reports it and the
    # next check is clean again
    bad = U.copy()
    bad[0, 17] = -1.0
    mesh.residual(torch.from_numpy(bad).cuda())
    with pytest.raises(h.HfdError) as e:
        mesh.check()
    assert e.value.status == 6
    mesh.check()


def test_3d_argument_validation(box):
    h = _cuda()
    m, P = box
    mesh = h.Mesh3(m)
    with pytest.raises(h.HfdError):
        mesh.prep_set("vidx", mesh.prep_get("vidx"))            # connectivity is read-only
    with pytest.raises(h.HfdError):
        mesh.prep_set("w5", np.zeros(7))                        # wrong count
    bad = mesh.prep_get("sten")
    bad[5] = N ** 3
    with pytest.raises(h.HfdError):
        mesh.prep_set("sten", bad)                              # stencil id out of range
    U = torch.from_numpy(T.uniform_state3(m)).cuda()
    with pytest.raises(h.HfdError):
        mesh.steps(U, 0.0, 1)                                   # dt must be positive
    with pytest.raises(h.HfdError):
        h.Mesh3(dict(m, tet=np.where(m["tet"] == 3, N ** 3 + 5, m["tet"])))


def test_3d_divergence_lane_counts_agree(box):
    """1, 2 and 4 lanes per vertex in the divergence gather give the same residual and steps to
    rounding (each count deterministic: two runs are bit-identical)."""
    h = _cuda()
    m, P = box
    U = T.vortex_tube(m)
    mesh = h.Mesh3(m)
    out = {}
    for lanes in (1, 2, 4):
        mesh.set_lanes(lanes)
        R = _residual(mesh, U)
        assert np.array_equal(R, _residual(mesh, U))
        X = torch.from_numpy(U.copy()).cuda()
        mesh.steps(X, 0.01, 2)
        torch.cuda.synchronize()
        mesh.check()
        out[lanes] = (R, X.cpu().numpy())
    for lanes in (2, 4):
        assert max(_groups(out[lanes][0], out[1][0])) < 1e-13
        assert np.abs(out[lanes][1] - out[1][1]).max() < 1e-13 * np.abs(out[1][1]).max()
    with pytest.raises(h.HfdError):
        mesh.set_lanes(3)
