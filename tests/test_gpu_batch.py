"""GPU tests of batches (many meshes advanced together) and of the persistent launch."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2109_01286_gb300 as pkg
    return pkg


@pytest.fixture(scope="module")
def members():
    return synth.batched_vortices(n=3, seed=11, vmin=300, vmax=1500)


def _state(mesh, U):
    return mesh.import_state(torch.from_numpy(np.ascontiguousarray(U)).cuda())


def test_batch_residual_and_steps_equal_single_meshes(members):
    pkg = _pkg()
    preps = [pkg.Prep(x["mesh"]) for x in members]
    batch = pkg.Prep.concat(preps).upload()
    assert batch.stats.nmember == 3
    Ub = np.concatenate([x["U"] for x in members], axis=1)
    Rb = batch.export_state(batch.residual(_state(batch, Ub))).cpu().numpy()
    Xb = _state(batch, Ub)
    batch.steps(Xb, 0.0, 2)                                    # own CFL step per member
    Sb = batch.export_state(Xb).cpu().numpy()
    dts = batch.last_dt()
    off = 0
    for k, x in enumerate(members):
        single = preps[k].upload()
        V = x["U"].shape[1]
        R = single.export_state(single.residual(_state(single, x["U"]))).cpu().numpy()
        np.testing.assert_array_equal(Rb[:, off:off + V], R)
        X = _state(single, x["U"])
        single.steps(X, 0.0, 2)
        np.testing.assert_array_equal(Sb[:, off:off + V], single.export_state(X).cpu().numpy())
        assert dts[k] == single.last_dt()
        off += V
    assert len(set(dts)) == 3


def test_batch_adjoint_equals_single_mesh_adjoints(members):
    """hfd_adjoint on a batch (one fixed dt for every member) gives each member's own adjoint:
    the transposed gathers of the union mesh visit a member's rows in the member's order."""
    pkg = _pkg()
    preps = [pkg.Prep(x["mesh"]) for x in members]
    batch = pkg.Prep.concat(preps).upload()
    Ub = np.concatenate([x["U"] for x in members], axis=1)
    rng = np.random.default_rng(3)
    lams = [rng.standard_normal(x["U"].shape) for x in members]
    dt = 0.01                                 # below every member's CFL step (>= 0.037)
    Lb = batch.export_state(batch.adjoint(_state(batch, Ub), _state(batch, np.concatenate(lams, axis=1)),
                                          dt=dt)).cpu().numpy()
    off = 0
    for k, x in enumerate(members):
        single = preps[k].upload()
        V = x["U"].shape[1]
        L = single.export_state(single.adjoint(_state(single, x["U"]), _state(single, lams[k]),
                                               dt=dt)).cpu().numpy()
        err = np.abs(Lb[:, off:off + V] - L).max() / np.abs(L).max()
        assert err < 1e-13, (k, err)
        off += V


def test_batch_matches_oracle_residual(members):
    pkg = _pkg()
    x = members[0]
    P = oracle.prepare(x["mesh"])
    R_ref = oracle.residual(x["mesh"], P, x["U"].copy())
    batch = pkg.Prep.concat([pkg.Prep(y["mesh"]) for y in members]).upload()
    Ub = np.concatenate([y["U"] for y in members], axis=1)
    Rb = batch.export_state(batch.residual(_state(batch, Ub))).cpu().numpy()
    V = x["U"].shape[1]
    err = np.linalg.norm(Rb[:, :V] - R_ref) / np.linalg.norm(R_ref)
    assert err < 1e-7, err                    # full path (library coefficients), see parity tests


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_persistent_launch_equals_four_launch_stage(members, precision):
    """The persistent stage kernel runs the same per-entity code as the four separate kernels;
    the compiler may contract multiply-adds differently in the fused kernel, so the results
    agree to rounding of the path's precision."""
    pkg = _pkg()
    tol = 1e-12 if precision == "fp64" else 2e-6
    batch = pkg.Prep.concat([pkg.Prep(y["mesh"]) for y in members]).upload(precision)
    Ub = np.concatenate([y["U"] for y in members], axis=1)
    a = _state(batch, Ub)
    b = a.clone()
    batch.set_launch(False)
    batch.steps(a, 0.0, 2)
    batch.set_launch(True)
    batch.steps(b, 0.0, 2)
    torch.cuda.synchronize()
    batch.check()
    assert (torch.linalg.norm(a - b) / torch.linalg.norm(a)).item() < tol
    persistent, grid, lanes, staged = batch.autotune(_state(batch, Ub))
    assert persistent in (0, 1) and lanes in (1, 2, 4, 8) and staged in (0, 1)
    c = _state(batch, Ub)
    batch.steps(c, 0.0, 2)
    torch.cuda.synchronize()
    assert (torch.linalg.norm(a - c) / torch.linalg.norm(a)).item() < tol


def test_persistent_barrier_wait_gives_up_and_reports_timeout(members):
    """A barrier poll bound of zero makes every early-arriving block give up at once: the kernel
    ends, the error word says HFD_ERR_TIMEOUT, and the mesh works again afterwards."""
    pkg = _pkg()
    m = pkg.Prep(members[2]["mesh"]).upload()
    U = _state(m, members[2]["U"])
    m.set_launch(True, 0)
    m.set_barrier_limit(0)
    m.step(U.clone(), 0.01)
    with pytest.raises(pkg.HfdError) as e:
        m.check()
    assert e.value.status == 8
    m.set_barrier_limit(1 << 24)
    a = U.clone()
    m.step(a, 0.01)
    m.check()
    m.set_launch(False)
    b = U.clone()
    m.step(b, 0.01)
    torch.cuda.synchronize()
    assert (torch.linalg.norm(a - b) / torch.linalg.norm(a)).item() < 1e-12


@pytest.mark.parametrize("given_dt", [False, True])
def test_batch_api_with_one_array_per_member(members, given_dt):
    """hfd_batch_step: member states in their own input order, advanced together, equal each
    member's own mesh bit for bit, with each member's CFL step or with given steps."""
    pkg = _pkg()
    preps = [pkg.Prep(x["mesh"]) for x in members]
    batch = pkg.Batch(preps)
    states = [torch.from_numpy(np.ascontiguousarray(x["U"])).cuda() for x in members]
    dts = [2e-3, 3e-3, 1e-3] if given_dt else None
    for _ in range(2):
        batch.step(states, dts)
    got_dt = batch.last_dt()
    for k, x in enumerate(members):
        single = preps[k].upload()
        X = _state(single, x["U"])
        for _ in range(2):
            single.step(X, dts[k] if given_dt else 0.0)
        np.testing.assert_array_equal(states[k].cpu().numpy(), single.export_state(X).cpu().numpy())
        assert got_dt[k] == (dts[k] if given_dt else single.last_dt())
    with pytest.raises(pkg.HfdError):
        batch.step(states, [1e-3, 0.0, 1e-3])
