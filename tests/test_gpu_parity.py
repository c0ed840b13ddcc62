"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Two kinds of comparison:
  * kernel parity -- the library's host preprocessing is run, its geometry coefficients are
    replaced by the oracle's (after checking that both made the same discrete choices), and the
    GPU residual / step must match the oracle to relative L2 1e-12 per row group;
  * full-path parity -- the library's own coefficients.  Its 5-node weights come from a
    different SVD than numpy's and truncated pseudo-inverses with small retained singular
    values are sensitive to rounding (up to ~1e-7 on a few stencils), so the bar is looser and
    stated per test.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import (elementwise_rel, inject_oracle_coefficients, near_threshold_vertices,
                         oracle_blocks, rel_l2_groups)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-12
# element-wise bound (|R - R_ref| / (|R_ref| + rms of the row group), every entry) of the FP64
# kernel-parity tests
EL_FP64 = 1e-11


def _hfd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2109_01286_gb300 as pkg
    return pkg


def _residual(mesh, U):
    Ui = mesh.import_state(torch.from_numpy(U).cuda())
    R = mesh.export_state(mesh.residual(Ui))
    torch.cuda.synchronize()
    return R.cpu().numpy()


@pytest.fixture(scope="module")
def c1():
    m = synth.jittered_grid(40, 40, 10.0, 10.0, seed=1)
    P = oracle.prepare(m)
    U = synth.isentropic_vortex(m)
    return m, P, U


@pytest.fixture(scope="module")
def quad():
    m = synth.jittered_box_with_ghosts(40, 40, (0.0, 1.0), (0.0, 1.0), 5, seed=2)
    P = oracle.prepare(m)
    U = synth.four_quadrant(m)
    return m, P, U


def _kernel_mesh(pkg, m, P, **opts):
    prep = pkg.Prep(m, **opts)
    inject_oracle_coefficients(prep, P, len(m["x"]))
    return prep.upload()


def test_residual_kernel_parity_fp64_vortex(c1):
    pkg = _hfd()
    m, P, U = c1
    mesh = _kernel_mesh(pkg, m, P)
    R = _residual(mesh, U)
    R_ref = oracle.residual(m, P, U.copy())
    err = rel_l2_groups(R, R_ref)
    assert max(err) < TOL_FP64, err
    assert elementwise_rel(R, R_ref) < EL_FP64


def test_residual_full_path_fp64_vortex(c1):
    pkg = _hfd()
    m, P, U = c1
    mesh = pkg.Mesh(m)
    R = _residual(mesh, U)
    R_ref = oracle.residual(m, P, U.copy())
    err = rel_l2_groups(R, R_ref)
    # the library's own coefficients: their gap to the oracle's follows from each stencil's
    # condition number (see the library-coefficient test below); ~2e-11 here
    assert max(err) < 1e-10, err
    assert elementwise_rel(R, R_ref) < 1e-9


@pytest.mark.parametrize("case", ["c1", "quad"])
def test_residual_full_path_fp64_on_library_coefficients(case, request):
    """The full FP64 path (the library's own preprocessing) against the oracle's residual
    evaluated with those same coefficients: the method's arithmetic agrees to 1e-12 in L2 and
    element-wise.  The coefficients themselves differ from the oracle's by at most a few units
    of eps times each stencil's condition number (tests/test_native_cpu.py), which is the whole
    of the remaining full-path gap."""
    from gpu_helpers import oracle_with_library_coefficients, elementwise_rel
    pkg = _hfd()
    m, P, U = request.getfixturevalue(case)
    prep = pkg.Prep(m)
    Q = oracle_with_library_coefficients(P, prep)
    R = _residual(prep.upload("fp64"), U)
    R_ref = oracle.residual(m, Q, U.copy())
    keep = P.active
    if case == "quad":
        keep = np.setdiff1d(P.active, near_threshold_vertices(m, Q, U, Q.opts))
    assert max(rel_l2_groups(R, R_ref, keep)) < 1e-12
    assert elementwise_rel(R, R_ref, keep) < 1e-10


def test_residual_kernel_parity_fp64_four_quadrant(quad):
    """Shocks and contacts: the WENO 3-node branch and the transmissive ghosts are exercised."""
    pkg = _hfd()
    m, P, U = quad
    mesh = _kernel_mesh(pkg, m, P)
    R = _residual(mesh, U)
    R_ref = oracle.residual(m, P, U.copy())
    d = {}
    oracle.hfd_oracle.edge_values(P, U.copy(), P.opts, d)
    assert sum(int((~s).sum()) for s in d["smooth"]) > 100      # the 3-node branch is used
    bad = near_threshold_vertices(m, P, U, P.opts)
    keep = np.setdiff1d(P.active, bad)
    assert len(keep) > 0.95 * len(P.active)
    err = rel_l2_groups(R, R_ref, keep)
    assert max(err) < TOL_FP64, err
    assert elementwise_rel(R, R_ref, keep) < EL_FP64
    assert np.all(R[:, m["ghost_ids"]] == 0.0)


def test_step_kernel_parity_fp64(c1):
    pkg = _hfd()
    m, P, U = c1
    mesh = _kernel_mesh(pkg, m, P)
    dt = oracle.cfl_dt(m, P, U)
    ref = oracle.step(m, P, U, dt)
    Ui = mesh.import_state(torch.from_numpy(U).cuda())
    mesh.step(Ui, dt)
    out = mesh.export_state(Ui).cpu().numpy()
    err = rel_l2_groups(out - U, ref - U)            # compare the increments
    assert max(err) < 1e-11, err
    mesh.check()


def test_step_kernel_parity_with_ghosts(quad):
    pkg = _hfd()
    m, P, U = quad
    mesh = _kernel_mesh(pkg, m, P)
    dt = 0.5 * oracle.cfl_dt(m, P, U)
    ref = oracle.step(m, P, U, dt)
    Ui = mesh.import_state(torch.from_numpy(U).cuda())
    mesh.step(Ui, dt)
    out = mesh.export_state(Ui).cpu().numpy()
    bad = near_threshold_vertices(m, P, U, P.opts)
    keep = np.setdiff1d(P.active, bad)
    err = rel_l2_groups(out - U, ref - U, keep)
    assert max(err) < 1e-11, err
    # ghosts refreshed from their donors at the end of the step
    g, dn = m["ghost_ids"], m["ghost_donor"]
    np.testing.assert_array_equal(out[0:4, g], out[0:4, dn])


def test_device_time_step_matches_oracle(c1):
    pkg = _hfd()
    m, P, U = c1
    mesh = pkg.Mesh(m)
    Ui = mesh.import_state(torch.from_numpy(U).cuda())
    mesh.step(Ui, 0.0)
    assert abs(mesh.last_dt() - oracle.cfl_dt(m, P, U)) < 1e-15 * oracle.cfl_dt(m, P, U)


def test_graph_replay_and_host_form_equal_direct_steps(c1):
    pkg = _hfd()
    m, P, U = c1
    mesh = pkg.Mesh(m)
    dt = 0.02
    a = mesh.import_state(torch.from_numpy(U).cuda())
    b = a.clone()
    for _ in range(3):
        mesh.step(a, dt)
    mesh.steps(b, dt, 3)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    hin = torch.from_numpy(U.copy()).pin_memory()
    hout = torch.empty_like(hin).pin_memory()
    mesh.steps_host(hin, hout, dt, 3)
    np.testing.assert_array_equal(hout.numpy(), mesh.export_state(a).cpu().numpy())


def test_renumbering_does_not_change_results(c1):
    pkg = _hfd()
    m, P, U = c1
    R1 = _residual(pkg.Mesh(m, renumber=True), U)
    R0 = _residual(pkg.Mesh(m, renumber=False), U)
    np.testing.assert_array_equal(R0, R1)


def test_viscous_kernel_parity_taylor_green():
    pkg = _hfd()
    n = 24
    m = synth.jittered_grid(n, n, 2 * np.pi, 2 * np.pi, seed=3)
    mach = 0.1
    p0 = 1.0 / (1.4 * mach * mach)
    kw = dict(viscous=True, mu=0.01, R_gas=p0)
    P = oracle.prepare(m, oracle.Options(**kw))
    U = synth.taylor_green(m, mach=mach)
    mesh = _kernel_mesh(pkg, m, P, **kw)
    R = _residual(mesh, U)
    R_ref = oracle.residual(m, P, U.copy())
    err = rel_l2_groups(R, R_ref)
    assert max(err) < 1e-11, err
    assert elementwise_rel(R, R_ref) < 10 * EL_FP64


def test_fp32_bulk_error_against_fp64_oracle(c1):
    """FP32-bulk path: interpolation, fluxes and divergence in FP32; state, RK combination,
    geometry solves and WENO weight ratios in FP64.  Its residual error is stated, not zero."""
    pkg = _hfd()
    m, P, U = c1
    prep = pkg.Prep(m, precision="fp32")
    inject_oracle_coefficients(prep, P, len(m["x"]))
    R = _residual(prep.upload(), U)
    R_ref = oracle.residual(m, P, U.copy())
    err = rel_l2_groups(R, R_ref)
    assert max(err) < 1e-4, err


def test_error_word_reports_nonfinite_state(c1):
    pkg = _hfd()
    m, P, U = c1
    mesh = pkg.Mesh(m)
    Ub = U.copy()
    Ub[0, 7] = np.nan
    Ui = mesh.import_state(torch.from_numpy(Ub).cuda())
    mesh.step(Ui, 0.01)
    with pytest.raises(pkg.HfdError) as ei:
        mesh.check()
    assert ei.value.status == 6
    mesh.check()                                      # the word was cleared


@pytest.mark.parametrize("precision,tol,margin", [("fp64", TOL_FP64, 1e-9), ("fp32", 1e-4, 1e-3)])
def test_full_size_four_quadrant_sampled_vertices(precision, tol, margin):
    """The 1024 x 1024 four-quadrant workload (5 ghost layers) in the bench's configuration,
    FP64 and FP32 bulk: GPU residual at sampled vertices against the FP64 oracle computed one
    vertex at a time, with the oracle's coefficients substituted for the sampled vertices'
    stencils.  FP32 decides the WENO branch on FP32 data, so its near-threshold margin is wider."""
    pkg = _hfd()
    n = 1024
    m = synth.jittered_box_with_ghosts(n, n, (0.0, 1.0), (0.0, 1.0), 5, seed=2)
    U = synth.four_quadrant(m)
    V = len(m["x"])
    rng = np.random.default_rng(0)
    topo = oracle.build_topology(m)
    act = np.nonzero(~topo["ghost"])[0]
    # sample near the centre (shocks), near the boundary (ghosts) and uniformly
    xy = np.stack([m["x"], m["y"]], 1)
    near_c = act[np.linalg.norm(xy[act] - 0.5, axis=1) < 0.01]
    near_b = act[(np.minimum(xy[act], 1 - xy[act]).min(axis=1)) < 0.003]
    samples = np.unique(np.concatenate([rng.choice(near_c, 4, replace=False),
                                        rng.choice(near_b, 4, replace=False),
                                        rng.choice(act, 4, replace=False)]))
    P = oracle.prepare(m, active=samples, topo=topo)
    R_ref = oracle.residual(m, P, U.copy())
    prep = pkg.Prep(m)
    fe = prep.get("flux_edges")
    pos = np.searchsorted(fe, P.edges)
    assert np.array_equal(fe[pos], P.edges)
    assert np.array_equal(prep.get("stencil").reshape(-1, 6)[pos], P.stencil)
    w5 = prep.get("w5").reshape(-1, 2, 15)
    w3 = prep.get("w3").reshape(-1, 2, 3, 3)
    w5[pos], w3[pos] = P.w5, P.w3
    prep.set("w5", w5)
    prep.set("w3", w3)
    active = prep.get("active")
    vptr, eptr = prep.get("div_vptr"), prep.get("div_eptr")
    cptr = np.concatenate([[0], np.cumsum(3 * (2 * np.diff(vptr) + np.diff(eptr)))])
    coef = prep.get("div_coef")
    blocks = oracle_blocks(P, V)["div_coef"]
    off = 0
    for r, v in enumerate(P.active):
        k = np.searchsorted(active, v)
        ln = cptr[k + 1] - cptr[k]
        coef[cptr[k]:cptr[k + 1]] = blocks[off:off + ln]
        off += ln
    prep.set("div_coef", coef)
    mesh = prep.upload(precision)
    R = _residual(mesh, U)
    bad = near_threshold_vertices(m, P, U, P.opts, margin=margin)
    keep = np.setdiff1d(samples, bad)
    assert len(keep) >= 8
    # away from the discontinuities the exact residual is zero; there the floor is the
    # round-off scale of the divergence sums: |F| / h for the w rows (d_0 ~ 1/h) and
    # |F| / h^2 for the derivative rows (d_x, d_y ~ 1/h^2)
    F, _ = oracle.euler_flux(U[:4], 1.4)
    inv_h = n - 1
    # (FP32: 80-term sums of FP32 products, |error| <~ 80 * 2^-24 * |F| / h, so 1e-5 |F| / h)
    fl = TOL_FP64 if precision == "fp64" else 1e-5
    floors = [fl * np.abs(F).max() * inv_h, fl * np.abs(F).max() * inv_h ** 2]
    for v in keep:
        for g, rows in enumerate((slice(0, 4), slice(4, 12))):
            diff = np.linalg.norm(R[rows, v] - R_ref[rows, v])
            assert diff < tol * np.linalg.norm(R_ref[rows, v]) + floors[g], (v, g, diff)


def _fp64_branches(stencil, normal, U, opts, chunk=250000):
    """Alg. 1's branch per flux edge, side and characteristic component decided in FP64 by the
    oracle's own functions (Roe average, left eigenvectors, uniform WENO5 weights, Eq.
    (2d_hweno_intp)), on given stencils: (bits as in hfd_edge_branches, distance of omega_1 to
    the nearer threshold)."""
    from oracle import hfd_oracle as H
    bits = np.zeros(len(stencil), dtype=np.uint8)
    dist = np.zeros(len(stencil))
    for a in range(0, len(stencil), chunk):
        st = stencil[a:a + chunk]
        W = U[0:4][:, st]                                     # (4, n, 6)
        u, v, Hh, c = H.roe_average(W[:, :, 2], W[:, :, 3], opts.gamma)
        L, _ = H.eigenvectors(u, v, Hh, c, normal[a:a + chunk, 0], normal[a:a + chunk, 1],
                              opts.gamma)
        C = np.einsum("eij,jek->eik", L, W)                   # (n, 4, 6)
        b = np.zeros(len(st), dtype=np.uint8)
        d = np.full(len(st), np.inf)
        for side, order in enumerate([H.LEFT_ORDER, H.RIGHT_ORDER]):
            o1 = H.weno_weights(*[C[:, :, k] for k in order], opts.weno_eps)[0]   # (n, 4)
            rough = ~((o1 > opts.sens_lo) & (o1 < opts.sens_hi))
            for q in range(4):
                b |= (rough[:, q].astype(np.uint8) << (side * 4 + q))
            d = np.minimum(d, np.minimum(np.abs(o1 - opts.sens_lo), np.abs(o1 - opts.sens_hi)).min(1))
        bits[a:a + chunk] = b
        dist[a:a + chunk] = d
    return bits, dist


def test_fp64_path_sensor_decisions_equal_fp64_decisions_at_full_size():
    """The FP64 edge kernel takes Alg. 1's decision in FP32 and re-takes it in FP64 only inside
    a guard band around the thresholds.  Over every side and characteristic component of the
    full 1024 x 1024 four-quadrant mesh, on the initial state and on the state after two
    steps, its decisions must equal decisions taken entirely in FP64 (up to sensor values
    within 1e-9 of a threshold, where FP64 rounding order itself decides)."""
    pkg = _hfd()
    n = 1024
    m = synth.jittered_box_with_ghosts(n, n, (0.0, 1.0), (0.0, 1.0), 5, seed=2)
    prep = pkg.Prep(m)
    mesh = prep.upload("fp64")
    stencil = prep.get("stencil").reshape(-1, 6)
    normal = prep.get("normal").reshape(-1, 2)
    opts = oracle.Options()
    Ui = mesh.import_state(torch.from_numpy(synth.four_quadrant(m)).cuda())
    report = []
    for nsteps in (0, 2):
        X = Ui.clone()
        if nsteps:
            mesh.steps(X, 0.0, nsteps)
        gpu = mesh.edge_branches(X)
        U = mesh.export_state(X).cpu().numpy()
        assert np.all(np.isfinite(U)), nsteps          # the method's growth has not set in yet
        ref, dist = _fp64_branches(stencil, normal, U, opts)
        clear = dist > 1e-9
        mismatch = int(np.count_nonzero((gpu != ref) & clear))
        weno_sides = int(sum(np.count_nonzero(ref & (1 << k)) for k in range(8)))
        report.append((nsteps, mismatch, weno_sides, int(np.count_nonzero(~clear))))
        assert weno_sides > 1000, report
        assert mismatch == 0, report
    mesh.check()


def test_full_four_quadrant_256_residual_at_every_vertex(tmp_path):
    """The whole four-quadrant residual on a 256 x 256 mesh (65,536 physical vertices, the bench
    workload's structure at a size the oracle covers), every vertex and every row: the FP64 full
    path against the oracle's residual on the library's coefficients, element-wise and in L2.
    The oracle runs in spawned CPU workers over chunks of the active vertices, each with the
    oracle's own stencils and two-level sets (checked equal to the library's)."""
    import multiprocessing as mp
    import os
    from gpu_helpers import c2_chunk_oracle_residual, elementwise_rel
    pkg = _hfd()
    n = 256
    m = synth.jittered_box_with_ghosts(n, n, (0.0, 1.0), (0.0, 1.0), 5, seed=2)
    U = synth.four_quadrant(m)
    prep = pkg.Prep(m)
    lib_path = str(tmp_path / "lib.npz")
    np.savez(lib_path, **{k: prep.get(k) for k in ("flux_edges", "w5", "w3", "stencil", "active",
                                                   "div_vptr", "div_eptr", "div_coef")})
    R = _residual(prep.upload("fp64"), U)
    act = prep.get("active")
    chunks = np.array_split(act, 16)
    workers = max(1, min(16, len(os.sched_getaffinity(0))))
    with mp.get_context("spawn").Pool(workers) as pool:
        res = pool.map(c2_chunk_oracle_residual, [(n, c, lib_path) for c in chunks])
    R_ref = np.zeros_like(R)
    bad = []
    for chunk, Rc, b in res:
        R_ref[:, chunk] = Rc
        bad.append(b)
    keep = np.setdiff1d(act, np.concatenate(bad))
    assert len(keep) > 0.99 * len(act)
    assert max(rel_l2_groups(R, R_ref, keep)) < 1e-12
    assert elementwise_rel(R, R_ref, keep) < 1e-10


def test_vortex_trajectory_parity_20_steps(c1):
    """The 40 x 40 isentropic-vortex workload: 20 SSP-RK3 steps at CFL 0.3 (device time step)
    against the oracle's 20 steps (its own CFL step each time), with the oracle's coefficients
    (kernel parity); also the density error against the exact translated vortex."""
    pkg = _hfd()
    m, P, U = c1
    mesh = _kernel_mesh(pkg, m, P)
    X = mesh.import_state(torch.from_numpy(U).cuda())
    ref = U.copy()
    t = 0.0
    for _ in range(20):
        dt = oracle.cfl_dt(m, P, ref)
        ref = oracle.step(m, P, ref, dt)
        mesh.step(X, 0.0)
        assert abs(mesh.last_dt() - dt) <= 1e-12 * dt
        t += dt
    out = mesh.export_state(X).cpu().numpy()
    err = rel_l2_groups(out, ref)
    assert max(err) < 1e-10, err
    exact = synth.isentropic_vortex(m, t=t)
    l2 = np.sqrt(np.mean((out[0] - exact[0]) ** 2))
    assert l2 < 5e-3, l2


@pytest.mark.parametrize("precision,lanes,tol", [("fp64", 2, 1e-13), ("fp64", 8, 1e-13),
                                                 ("fp32", 1, 1e-4), ("fp32", 8, 1e-4)])
def test_divergence_lane_counts_agree(c1, precision, lanes, tol):
    """Every lanes-per-vertex variant of the divergence (different reduction orders) gives the
    default variant's residual to rounding."""
    pkg = _hfd()
    m, P, U = c1
    mesh = pkg.Prep(m).upload(precision)
    R0 = _residual(mesh, U)
    mesh.set_lanes(lanes)
    R1 = _residual(mesh, U)
    assert np.linalg.norm(R1 - R0) <= tol * np.linalg.norm(R0)


@pytest.mark.parametrize("case", ["vortex", "quad", "tgv_viscous", "circle", "torus3", "batch"])
def test_staged_fp32_divergence_equals_unstaged_at_eight_lanes(case):
    """The staged FP32 divergence (tiles of vertices whose coefficient and index chunks are
    bulk-copied into shared memory, double-buffered) sums each vertex's entries in the order of
    the unstaged kernel at 8 lanes: residuals and graph-replayed steps are bit-identical,
    on meshes of one tile or fewer (3x3 torus), with ghosts, viscous rows, a Delaunay mesh and a
    batch of uneven meshes."""
    pkg = _hfd()
    visc = dict(viscous=True, mu=0.01, prandtl=0.72, R_gas=1.0 / (1.4 * 0.01))
    kw = {}
    if case == "vortex":
        m = synth.jittered_grid(40, 40, 10.0, 10.0, seed=1)
        U = synth.isentropic_vortex(m)
    elif case == "quad":
        m = synth.jittered_box_with_ghosts(48, 48, (0.0, 1.0), (0.0, 1.0), 5, seed=2)
        U = synth.four_quadrant(m)
    elif case == "tgv_viscous":
        m = synth.jittered_grid(32, 32, 2 * np.pi, 2 * np.pi, seed=3)
        U = synth.taylor_green(m)
        kw = visc
    elif case == "circle":
        m = synth.embedded_circle_box(24, seed=8)
        U = synth.circular_sod(m)
    elif case == "torus3":
        m = synth.jittered_grid(3, 3, 10.0, 10.0, seed=1)
        U = synth.isentropic_vortex(m)
    if case == "batch":
        members = synth.batched_vortices(n=6, seed=4, vmin=300, vmax=3000)
        mesh = pkg.Prep.concat([pkg.Prep(x["mesh"]) for x in members]).upload("fp32")
        U = np.concatenate([x["U"] for x in members], axis=1)
    else:
        mesh = pkg.Mesh(m, precision="fp32", **kw)
    Ui = mesh.import_state(torch.from_numpy(U).cuda())
    nsteps = 1 if case == "quad" else 3          # the four-quadrant state grows fast (the method)
    out = {}
    for staged in (1, 0):
        mesh.set_div_staged(staged)
        mesh.set_lanes(8)
        R = mesh.residual(Ui.clone())
        X = Ui.clone()
        mesh.steps(X, 0.0, nsteps)
        torch.cuda.synchronize()
        mesh.check()
        out[staged] = (R, X)
    assert torch.isfinite(out[1][0]).all() and torch.isfinite(out[1][1]).all()
    assert torch.equal(out[1][0], out[0][0])
    assert torch.equal(out[1][1], out[0][1])


@pytest.mark.parametrize("case", ["vortex", "quad", "tgv_viscous", "circle", "batch"])
def test_folded_double_float_divergence_equals_plain_fp64(case):
    """The FP64 divergence in folded double-float form (edge-row endpoint averages folded into
    the vertex rows, centre-vertex differences, products on the FP32 pipe) against the plain FP64
    form: residuals and three graph-replayed steps agree to 1e-12 in L2 (1e-11 element-wise) on
    smooth and shock data, with ghosts, a Delaunay mesh and a batch, and to 3e-11 on the
    low-Mach viscous Taylor-Green state."""
    from gpu_helpers import elementwise_rel
    pkg = _hfd()
    visc = dict(viscous=True, mu=0.01, prandtl=0.72, R_gas=1.0 / (1.4 * 0.01))
    kw = {}
    if case == "vortex":
        m = synth.jittered_grid(48, 48, 10.0, 10.0, seed=1)
        U = synth.isentropic_vortex(m)
    elif case == "quad":
        m = synth.jittered_box_with_ghosts(48, 48, (0.0, 1.0), (0.0, 1.0), 5, seed=2)
        U = synth.four_quadrant(m)
    elif case == "tgv_viscous":
        m = synth.jittered_grid(32, 32, 2 * np.pi, 2 * np.pi, seed=3)
        U = synth.taylor_green(m)
        kw = visc
    elif case == "circle":
        m = synth.embedded_circle_box(24, seed=8)
        U = synth.circular_sod(m)
    if case == "batch":
        members = synth.batched_vortices(n=6, seed=4, vmin=300, vmax=3000)
        mesh = pkg.Prep.concat([pkg.Prep(x["mesh"]) for x in members]).upload("fp64")
        U = np.concatenate([x["U"] for x in members], axis=1)
    else:
        mesh = pkg.Mesh(m, **kw)
    Ui = mesh.import_state(torch.from_numpy(U).cuda())
    out = {}
    for folded in (1, 0):
        mesh.set_fp64_div(folded)
        R = mesh.residual(Ui.clone()).cpu().numpy()
        X = Ui.clone()
        mesh.steps(X, 0.0, 1 if case == "quad" else 3)
        torch.cuda.synchronize()
        mesh.check()
        out[folded] = (R, X.cpu().numpy())
    # low Mach number: the energy flux's nearly divergence-free part, (E + p) u with E + p about
    # 250 at Mach 0.1, cancels in every row, and the 48-bit products of the folded form show
    # through (measured 1.2e-11 before rounding the split's low part, CPU emulation against an
    # extended-precision sum: folded 1.2e-11, plain FP64 8e-13)
    tol = 3e-11 if case == "tgv_viscous" else 1e-12
    R1, R0 = out[1][0], out[0][0]
    assert max(rel_l2_groups(R1, R0)) < tol
    assert elementwise_rel(R1, R0) < 10 * tol
    X1, X0 = out[1][1], out[0][1]
    assert max(rel_l2_groups(X1 - U[:, mesh.perm], X0 - U[:, mesh.perm])) < 10 * tol


def test_folded_divergence_is_for_fp64_meshes(c1):
    pkg = _hfd()
    m, P, U = c1
    mesh = pkg.Mesh(m, precision="fp32")
    with pytest.raises(pkg.HfdError) as e:
        mesh.set_fp64_div(1)
    assert e.value.status == 9
    mesh.set_fp64_div(0)


@pytest.mark.parametrize("case", ["vortex", "quad", "circle", "torus3", "batch"])
def test_gather_staged_fp32_divergence_equals_unstaged_at_four_lanes(case):
    """The gather-staged FP32 divergence (each block's distinct vertex and edge fluxes copied
    once into shared memory, 16-bit tile-local indices) runs the unstaged kernel's chunk loop:
    residuals and graph-replayed steps are bit-identical to the unstaged kernel at 4 lanes, on
    meshes of one partial tile (3x3 torus), with ghosts, a Delaunay mesh and a batch."""
    pkg = _hfd()
    if case == "vortex":
        m = synth.jittered_grid(40, 40, 10.0, 10.0, seed=1)
        U = synth.isentropic_vortex(m)
    elif case == "quad":
        m = synth.jittered_box_with_ghosts(48, 48, (0.0, 1.0), (0.0, 1.0), 5, seed=2)
        U = synth.four_quadrant(m)
    elif case == "circle":
        m = synth.embedded_circle_box(24, seed=8)
        U = synth.circular_sod(m)
    elif case == "torus3":
        m = synth.jittered_grid(3, 3, 10.0, 10.0, seed=1)
        U = synth.isentropic_vortex(m)
    if case == "batch":
        members = synth.batched_vortices(n=6, seed=4, vmin=300, vmax=3000)
        mesh = pkg.Prep.concat([pkg.Prep(x["mesh"]) for x in members]).upload("fp32")
        U = np.concatenate([x["U"] for x in members], axis=1)
    else:
        mesh = pkg.Mesh(m, precision="fp32")
    Ui = mesh.import_state(torch.from_numpy(U).cuda())
    nsteps = 1 if case == "quad" else 3
    out = {}
    for staged in (2, 0):
        mesh.set_div_staged(staged)
        mesh.set_lanes(4)
        R = mesh.residual(Ui.clone())
        X = Ui.clone()
        mesh.steps(X, 0.0, nsteps)
        torch.cuda.synchronize()
        mesh.check()
        out[staged] = (R, X)
    assert torch.isfinite(out[2][0]).all() and torch.isfinite(out[2][1]).all()
    assert torch.equal(out[2][0], out[0][0])
    assert torch.equal(out[2][1], out[0][1])


def test_gather_staged_divergence_is_for_inviscid_fp32_meshes(c1):
    pkg = _hfd()
    m, P, U = c1
    for kw in ({}, {"precision": "fp32", "viscous": True, "mu": 0.01, "R_gas": 1.0}):
        mesh = pkg.Mesh(m, **kw)
        with pytest.raises(pkg.HfdError) as e:
            mesh.set_div_staged(2)
        assert e.value.status == 9
        mesh.set_div_staged(0)
    with pytest.raises(pkg.HfdError):
        pkg.Mesh(m, precision="fp32").set_div_staged(3)


def test_staged_divergence_is_for_fp32_meshes(c1):
    pkg = _hfd()
    m, P, U = c1
    mesh = pkg.Mesh(m)
    with pytest.raises(pkg.HfdError) as e:
        mesh.set_div_staged(1)
    assert e.value.status == 9
    mesh.set_div_staged(0)


def test_viscous_steps_parity_taylor_green():
    """Three SSP-RK3 steps of the viscous Taylor-Green workload (24 x 24 periodic, Mach 0.1,
    mu 0.01) with a fixed step, through the graph-replayed stage path, against the oracle's
    three steps (kernel parity)."""
    pkg = _hfd()
    n = 24
    m = synth.jittered_grid(n, n, 2 * np.pi, 2 * np.pi, seed=3)
    mach = 0.1
    p0 = 1.0 / (1.4 * mach * mach)
    kw = dict(viscous=True, mu=0.01, R_gas=p0)
    opts = oracle.Options(**kw)
    P = oracle.prepare(m, opts)
    U = synth.taylor_green(m, mach=mach)
    h = 2 * np.pi / n
    dt = 0.3 * h / (1.0 + np.sqrt(1.4 * p0))
    mesh = _kernel_mesh(pkg, m, P, **kw)
    X = mesh.import_state(torch.from_numpy(U).cuda())
    ref = U.copy()
    for _ in range(3):
        ref = oracle.step(m, P, ref, dt, opts)
        mesh.steps(X, dt, 1)
    out = mesh.export_state(X).cpu().numpy()
    err = rel_l2_groups(out, ref)
    assert max(err) < 1e-11, err


def test_caller_allocator_holds_the_mesh_and_gives_identical_results(c1):
    """hfd_options.dev_alloc / dev_free with PyTorch's caching allocator: the mesh's device
    blocks are counted by torch, released on destroy, and the results are bit-identical."""
    import gc
    pkg = _hfd()
    m, P, U = c1
    a = pkg.Mesh(m)
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    b = pkg.Mesh(m, allocator="torch")
    held = torch.cuda.memory_allocated() - before
    assert held >= b.stats.device_bytes > 0
    np.testing.assert_array_equal(_residual(a, U), _residual(b, U))
    Xa = a.import_state(torch.from_numpy(U).cuda())
    Xb = b.import_state(torch.from_numpy(U).cuda())
    a.steps(Xa, 0.0, 3)
    b.steps(Xb, 0.0, 3)
    torch.testing.assert_close(Xa, Xb, rtol=0, atol=0)
    lam = torch.ones_like(Xa)
    dt = a.last_dt()
    torch.testing.assert_close(a.adjoint(Xa, lam, dt=dt), b.adjoint(Xb, lam, dt=dt), rtol=0, atol=0)
    total = b.stats.device_bytes
    mid = torch.cuda.memory_allocated()
    del b
    gc.collect()
    torch.cuda.synchronize()
    assert mid - torch.cuda.memory_allocated() >= total


@pytest.mark.parametrize("case", ["c1", "quad"])
def test_rusanov_residual_kernel_parity(case, request):
    """The alternative Riemann solver (hfd_options.flux = 1) against the oracle's Rusanov flux,
    FP64 kernel parity, on the vortex and on the four-quadrant mesh with ghosts."""
    pkg = _hfd()
    m, P, U = request.getfixturevalue(case)
    mesh = _kernel_mesh(pkg, m, P, flux="rusanov")
    R = _residual(mesh, U)
    opts = oracle.Options(flux="rusanov")
    R_ref = oracle.residual(m, P, U.copy(), opts)
    keep = np.setdiff1d(P.active, near_threshold_vertices(m, P, U, opts))
    err = rel_l2_groups(R, R_ref, keep)
    assert max(err) < TOL_FP64, err
    assert elementwise_rel(R, R_ref, keep) < EL_FP64
    R_roe = oracle.residual(m, P, U.copy())
    assert max(rel_l2_groups(R_roe, R_ref)) > 1e3 * TOL_FP64      # the solvers differ


def test_positivity_fallback_kernel_parity(c1):
    """R16 on a near-vacuum state: rho = p = 0.01 everywhere, random derivatives of size 0.05.
    The values are uniform, so every sensor decision is the 5-node branch, and the 5-node
    values overshoot below zero on about 6% of the sides.  Those sides fall back to the
    edge's end state, on the GPU as in the oracle."""
    pkg = _hfd()
    m, P, _ = c1
    rng = np.random.default_rng(17)
    U = synth.uniform_state(m, rho=0.01, p=0.01)
    U[4:] = 0.05 * rng.standard_normal(U[4:].shape)
    diag = {}
    R_ref = oracle.residual(m, P, U.copy(), diag=diag)
    assert 100 < diag["positivity_fallbacks"] < 0.5 * 2 * len(P.edges)
    R = _residual(_kernel_mesh(pkg, m, P), U)
    err = rel_l2_groups(R, R_ref)
    assert max(err) < TOL_FP64, err
    assert elementwise_rel(R, R_ref) < EL_FP64


@pytest.mark.parametrize("n", [3, 4, 5, 7, 9])
def test_tiny_periodic_mesh_kernel_parity(n):
    """Degenerate sizes: 3x3 to 9x9 tori (9 to 81 vertices, less than one thread block), where
    the two-level sets cover most or all of the mesh and the 6-node stencils wrap around it
    (below 7x7 a stencil spans more than half the period, so its minimum-image geometry is not
    the physical one; both sides take the same reading, and the case checks the indexing).
    Smooth random data; vertices whose sensor value lies within 1e-9 of a threshold are
    excluded."""
    pkg = _hfd()
    m = synth.jittered_grid(n, n, 1.0, 1.0, seed=9)
    P = oracle.prepare(m)
    rng = np.random.default_rng(19)
    U = synth.uniform_state(m)
    U[:4] *= 1.0 + 0.05 * rng.random((4, len(m["x"])))
    U[4:] = 0.05 * rng.standard_normal(U[4:].shape)
    R = _residual(_kernel_mesh(pkg, m, P), U)
    R_ref = oracle.residual(m, P, U.copy())
    keep = np.setdiff1d(P.active, near_threshold_vertices(m, P, U, P.opts))
    assert len(keep) > 0.8 * len(P.active)
    err = rel_l2_groups(R, R_ref, keep)
    assert max(err) < TOL_FP64, err
    assert elementwise_rel(R, R_ref, keep) < EL_FP64


@pytest.mark.parametrize("case", ["c1", "quad"])
def test_conservative_variant_kernel_parity(case, request):
    """hfd_options.conservative = 1 (median-dual value rows, dual-normal fluxes) against the
    oracle's conservative variant, FP64 kernel parity."""
    pkg = _hfd()
    m = request.getfixturevalue(case)[0]
    U = request.getfixturevalue(case)[2]
    opts = oracle.Options(conservative=True)
    P = oracle.prepare(m, opts)
    mesh = _kernel_mesh(pkg, m, P, conservative=True)
    R = _residual(mesh, U)
    R_ref = oracle.residual(m, P, U.copy(), opts)
    keep = np.setdiff1d(P.active, near_threshold_vertices(m, P, U, opts))
    assert len(keep) > 0.95 * len(P.active)
    err = rel_l2_groups(R, R_ref, keep)
    assert max(err) < TOL_FP64, err
    assert elementwise_rel(R, R_ref, keep) < EL_FP64


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-13), ("fp32", 1e-6)])
def test_conservative_variant_conserves_on_the_gpu(c1, precision, tol):
    """The library's own coefficients: on the periodic vortex mesh sum_v |C_v| R_v vanishes for
    the conserved rows, relative to sum_v |C_v| |R_v|, in FP64 and in FP32 bulk."""
    pkg = _hfd()
    m, _, U = c1
    prep = pkg.Prep(m, conservative=True)
    A = prep.get("dual_A")
    R = _residual(prep.upload(precision), U)
    total = (R[:4] * A).sum(axis=1)
    scale = (np.abs(R[:4]) * A).sum(axis=1)
    assert np.all(np.abs(total) < tol * scale), (total, scale)


def test_couette_channel_with_wall_bands_kernel_parity():
    """Sec. 3.2 Couette channel: x periodic, fixed ghost bands beyond both walls (donor -1)
    holding the exact solution, viscous (the paper's c_p = 10, kappa = 1/100, mu = 1/10).
    Residual and three SSP-RK3 steps through the graph path against the oracle (kernel parity);
    the ghost bands keep their values through the steps (every stage refreshes them from the
    step's input state)."""
    pkg = _hfd()
    R_gas = 0.4 * 10.0 / 1.4
    m = synth.couette_channel(16, 17, 6, seed=7)
    U = synth.couette(m)
    kw = dict(viscous=True, mu=0.1, prandtl=100.0, R_gas=R_gas)
    opts = oracle.Options(**kw)
    P = oracle.prepare(m, opts)
    mesh = _kernel_mesh(pkg, m, P, **kw)
    R = _residual(mesh, U)
    R_ref = oracle.residual(m, P, U.copy(), opts)
    scale = np.abs(oracle.euler_flux(U[:4], 1.4)[0]).max() / (10.0 / 16)
    assert np.abs(R - R_ref).max() < 1e-12 * scale
    dt = 0.2 * oracle.cfl_dt(m, P, U)
    X = mesh.import_state(torch.from_numpy(U).cuda())
    ref = U.copy()
    for _ in range(3):
        ref = oracle.step(m, P, ref, dt, opts)
        mesh.steps(X, dt, 1)
    out = mesh.export_state(X).cpu().numpy()
    # near the steady state the increments are tiny: compare the states to rounding
    for rows in (slice(0, 4), slice(4, 12)):
        assert np.abs(out[rows] - ref[rows]).max() <= 1e-13 * np.abs(U[rows]).max()
    g = m["ghost_ids"]
    np.testing.assert_array_equal(out[:, g], U[:, g])


def test_checkpoint_resume_continues_bit_identically(c1, tmp_path):
    """save_state / load_state: 4 steps straight equal 2 steps, a checkpoint to .npz, a reload
    into a new mesh and 2 more steps, bit for bit (CFL step each time)."""
    pkg = _hfd()
    m, _, U = c1
    a = pkg.Mesh(m)
    X = a.import_state(torch.from_numpy(U).cuda())
    a.steps(X, 0.0, 4)
    Y = a.import_state(torch.from_numpy(U).cuda())
    a.steps(Y, 0.0, 2)
    a.save_state(tmp_path / "ck.npz", Y, steps=np.int64(2))
    b = pkg.Mesh(m)
    Z, extra = b.load_state(tmp_path / "ck.npz")
    assert int(extra["steps"]) == 2
    b.steps(Z, 0.0, 2)
    np.testing.assert_array_equal(a.export_state(X).cpu().numpy(), b.export_state(Z).cpu().numpy())
    with pytest.raises(ValueError):
        pkg.Mesh(synth.jittered_grid(8, 8, 1.0, 1.0, seed=0)).load_state(tmp_path / "ck.npz")


@pytest.fixture(scope="module")
def csod():
    m = synth.embedded_circle_box(24, seed=8)
    P = oracle.prepare(m)
    U = synth.circular_sod(m)
    return m, P, U


def test_circular_sod_delaunay_mesh_kernel_parity(csod):
    """Sec. 3.3 circular Sod on the embedded-circle Delaunay mesh: residual and five SSP-RK3
    steps with the device CFL step against the oracle (kernel parity).  The discontinuity lies
    on a mesh line, so the WENO branch is taken all around the circle."""
    pkg = _hfd()
    m, P, U = csod
    mesh = _kernel_mesh(pkg, m, P)
    R = _residual(mesh, U)
    R_ref = oracle.residual(m, P, U.copy())
    d = {}
    oracle.hfd_oracle.edge_values(P, U.copy(), P.opts, d)
    assert sum(int((~s).sum()) for s in d["smooth"]) > 50
    bad = near_threshold_vertices(m, P, U, P.opts)
    keep = np.setdiff1d(P.active, bad)
    assert len(keep) > 0.95 * len(P.active)
    assert max(rel_l2_groups(R, R_ref, keep)) < TOL_FP64
    assert elementwise_rel(R, R_ref, keep) < EL_FP64
    X = mesh.import_state(torch.from_numpy(U).cuda())
    ref = U.copy()
    for _ in range(5):
        dt = oracle.cfl_dt(m, P, ref)
        ref = oracle.step(m, P, ref, dt)
        mesh.step(X, 0.0)
        assert abs(mesh.last_dt() - dt) <= 1e-12 * dt
    out = mesh.export_state(X).cpu().numpy()
    err = rel_l2_groups(out - U, ref - U)
    assert max(err) < 1e-10, err
    mesh.check()


@pytest.mark.parametrize("precision,margin,tol", [("fp64", 1e-5, 1e-6), ("fp32", 1e-3, 1e-4)])
def test_circular_sod_delaunay_mesh_full_path(csod, precision, margin, tol):
    """The library's own coefficients (and the FP32-bulk path) on the Delaunay mesh: residual
    against the oracle's.  Vertices reading an edge whose sensor lies within `margin` of a
    threshold are left out: the coefficient differences (FP64, up to ~1e-7 on a few truncated
    pseudo-inverses) or FP32 data may decide those branches either way."""
    pkg = _hfd()
    m, P, U = csod
    mesh = pkg.Mesh(m, precision=precision)
    R = _residual(mesh, U)
    R_ref = oracle.residual(m, P, U.copy())
    bad = near_threshold_vertices(m, P, U, P.opts, margin=margin)
    keep = np.setdiff1d(P.active, bad)
    assert len(keep) > 0.8 * len(P.active)
    err = rel_l2_groups(R, R_ref, keep)
    assert max(err) < tol, err


def test_lane_setter_and_autotuner_keep_results_to_rounding(c1):
    """hfd_mesh_set_lanes changes only the divergence's summation order; an invalid count is
    refused; the autotuner's pick (launch form, grid, lanes) steps to the default's rounding."""
    pkg = _hfd()
    m, P, U = c1
    mesh = pkg.Mesh(m)
    R1 = _residual(mesh, U)
    for lanes in (8, 2, 1):
        mesh.set_lanes(lanes)
        R = _residual(mesh, U)
        assert max(rel_l2_groups(R, R1)) < 1e-13, lanes
    with pytest.raises(pkg.HfdError) as e:
        mesh.set_lanes(3)
    assert e.value.status == 1
    Ui = mesh.import_state(torch.from_numpy(U).cuda())
    a = Ui.clone()
    mesh.steps(a, 0.0, 3)
    persistent, grid, lanes, staged = mesh.autotune(Ui)
    assert persistent in (0, 1) and lanes in (1, 2, 4, 8) and grid >= 0 and staged in (0, 1)
    b = Ui.clone()
    mesh.steps(b, 0.0, 3)
    torch.cuda.synchronize()
    mesh.check()
    assert (torch.linalg.norm(a - b) / torch.linalg.norm(a)).item() < 1e-12


def test_bounds_checked_build_runs_clean_and_matches(tmp_path):
    """The bounds-checked library (HFD_CHECKED=1: every gathered index of the forward kernels
    tested on the device) runs the residual and two steps of meshes covering every gather with
    a clean error word, and gives the normal build's results."""
    import json
    import os
    import subprocess
    import sys
    from gpu_helpers import run_checked_build_cases
    pkg = _hfd()
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = tmp_path / "checked.npz"
    code = (
        "import sys, numpy as np, torch\n"
        f"sys.path[:0] = [{root!r}, {os.path.join(root, 'tests')!r}]\n"
        "import paper_2109_01286_gb300 as pkg\n"
        "assert pkg.hfd.LIB_PATH.endswith('libhfd_check.so'), pkg.hfd.LIB_PATH\n"
        "from gpu_helpers import run_checked_build_cases\n"
        f"np.savez({str(out)!r}, **run_checked_build_cases(pkg, torch))\n")
    env = dict(os.environ, HFD_CHECKED="1")
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    ref = run_checked_build_cases(pkg, torch)
    got = np.load(out)
    diffs = {}
    for k, a in ref.items():
        b = got[k]
        diffs[k] = float(np.abs(a - b).max() / max(np.abs(a).max(), 1e-300))
        tol = 1e-6 if "fp32" in k else 1e-13
        assert diffs[k] <= tol, json.dumps(diffs)


@pytest.mark.parametrize("case,branch,precision,tol", [
    ("c1", "weno", "fp64", TOL_FP64), ("quad", "hermite", "fp64", TOL_FP64),
    ("quad", "weno", "fp64", TOL_FP64), ("c1", "weno", "fp32", 1e-4)])
def test_forced_branch_kernel_parity(case, branch, precision, tol, request):
    """Alg. 1 with one branch forced on every characteristic component and side (a testing
    aid): every edge of the smooth vortex through the WENO-weighted 3-node candidates, every
    edge of the four-quadrant problem through the 5-node values or the candidates; no branch is
    left to rounding, so no vertex is excluded."""
    pkg = _hfd()
    m, _, U = request.getfixturevalue(case)
    opts = oracle.Options(force_branch=branch)
    P = oracle.prepare(m, opts)
    prep = pkg.Prep(m, force_branch=branch, precision=precision)
    inject_oracle_coefficients(prep, P, len(m["x"]))
    R = _residual(prep.upload(), U)
    R_ref = oracle.residual(m, P, U.copy(), opts)
    err = rel_l2_groups(R, R_ref)
    assert max(err) < tol, err
    assert max(rel_l2_groups(R, oracle.residual(m, oracle.prepare(m), U.copy()))) > 10 * tol


def test_adjoint_refuses_a_forced_branch(c1):
    pkg = _hfd()
    m, _, U = c1
    mesh = pkg.Mesh(m, force_branch="weno")
    Ui = mesh.import_state(torch.from_numpy(U).cuda())
    with pytest.raises(pkg.HfdError) as e:
        mesh.adjoint(Ui, Ui.clone(), dt=0.01)
    assert e.value.status == 9


def test_circular_sod_against_radial_reference():
    """Sec. 3.3: the CUDA path's density on the embedded-circle meshes of 24 and 50 segments
    per side at t = 0.03 (fixed steps below CFL 0.3; the state of the method as read turns
    inadmissible soon after) against the high-resolution 1D radial reference solution, by the
    area-weighted L1 error over the physical vertices.  The error is that of the smeared
    shock, contact and rarefaction, and falls with the mesh."""
    from oracle import radial
    pkg = _hfd()
    T = 0.03
    rc, (rho_ref, _, _) = radial.circular_sod(T, n=4000)
    errs = []
    for n, k in ((24, 5), (50, 10)):
        m = synth.embedded_circle_box(n, seed=8)
        mesh = pkg.Mesh(m)
        X = mesh.import_state(torch.from_numpy(synth.circular_sod(m)).cuda())
        mesh.steps(X, T / k, k)
        mesh.check()
        rho = mesh.export_state(X)[0].cpu().numpy()
        phys = np.setdiff1d(np.arange(len(m["x"])), m["ghost_ids"])
        A = synth.vertex_areas(m)[phys]
        ref = np.interp(np.hypot(m["x"], m["y"])[phys], rc, rho_ref)
        errs.append(float(np.sum(A * np.abs(rho[phys] - ref)) / np.sum(A)))
    assert errs[0] < 0.025 and errs[1] < 0.016 and errs[1] < 0.8 * errs[0], errs


@pytest.mark.parametrize("flux", ["roe", "rusanov"])
@pytest.mark.parametrize("conservative", [False, True])
@pytest.mark.parametrize("viscous", [False, True])
def test_option_combinations_kernel_parity(flux, conservative, viscous):
    """Every combination of Riemann solver, conservative variant and viscous terms on the
    16-segment embedded-circle Delaunay mesh with the circular Sod state (ghost layers, WENO
    branch on the circle), residual kernel parity; vertices reading an edge whose sensor lies
    within 1e-9 of a threshold are excluded."""
    pkg = _hfd()
    m = synth.embedded_circle_box(16, seed=8)
    U = synth.circular_sod(m)
    kw = dict(flux=flux, conservative=conservative)
    if viscous:
        kw.update(viscous=True, mu=0.02, prandtl=0.72, R_gas=1.0)
    opts = oracle.Options(**kw)
    P = oracle.prepare(m, opts)
    R = _residual(_kernel_mesh(pkg, m, P, **kw), U)
    R_ref = oracle.residual(m, P, U.copy(), opts)
    keep = np.setdiff1d(P.active, near_threshold_vertices(m, P, U, opts))
    assert len(keep) > 0.9 * len(P.active)
    err = rel_l2_groups(R, R_ref, keep)
    assert max(err) < TOL_FP64, err
    assert elementwise_rel(R, R_ref, keep) < EL_FP64
