"""hfd_residual_static -- the residual for callers that cannot allocate device memory at call
time -- against hfd_residual, through the C ABI.

This file is collected last so that a run stopping at the first failure has already run every
other test.  It also passes when run alone in a fresh process: the entry point looks the fixed
scratch array up on every call, so the first call needs no preparation.

The static entry point runs the same kernels with the same launch shapes as hfd_residual, only
with its scratch moved into the fixed array, so the two results must be bit-identical.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2109_01286_gb300 as pkg
    return pkg


def test_static_scratch_residual_matches_allocating_entry_point():
    pkg = _pkg()
    m = synth.jittered_grid(40, 40, 10.0, 10.0, seed=1)            # 1,600 vertices
    mesh = pkg.Mesh(m)
    states = [synth.isentropic_vortex(m), synth.isentropic_vortex(m, beta=3.0, t=0.7)]
    for U in states:                                             # two calls in a row
        Ui = mesh.import_state(torch.from_numpy(U).cuda())
        R_ref = mesh.residual(Ui.clone())
        R = torch.full_like(Ui, float("nan"))
        mesh.residual_static(Ui.clone(), R)
        torch.cuda.synchronize()
        assert torch.isfinite(R).all()
        assert torch.equal(R, R_ref)


def test_static_scratch_residual_with_ghosts_and_fp32():
    pkg = _pkg()
    m = synth.jittered_box_with_ghosts(40, 40, (0.0, 1.0), (0.0, 1.0), 5, seed=2)
    U = synth.four_quadrant(m)
    for prec in ("fp64", "fp32"):
        mesh = pkg.Prep(m).upload(prec)
        Ui = mesh.import_state(torch.from_numpy(U).cuda())
        R_ref = mesh.residual(Ui.clone())
        for _ in range(2):
            R = torch.full_like(Ui, float("nan"))
            mesh.residual_static(Ui.clone(), R)
            torch.cuda.synchronize()
            assert torch.equal(R, R_ref), prec


def test_static_scratch_residual_viscous_on_a_side_stream():
    """A viscous mesh puts the viscous vertex fluxes between the inviscid fluxes and the edge
    fluxes inside the fixed array; the calls run on a stream other than the current one."""
    pkg = _pkg()
    m = synth.jittered_grid(24, 24, 2 * np.pi, 2 * np.pi, seed=3)
    U = synth.taylor_green(m)
    mesh = pkg.Mesh(m, viscous=True, mu=0.01, prandtl=0.72, R_gas=1.0 / (1.4 * 0.01))
    Ui = mesh.import_state(torch.from_numpy(U).cuda())
    R_ref = mesh.residual(Ui.clone())
    side = torch.cuda.Stream()
    torch.cuda.synchronize()
    for _ in range(2):
        R = torch.full_like(Ui, float("nan"))
        Uc = Ui.clone()
        torch.cuda.synchronize()
        mesh.residual_static(Uc, R, stream=side)
        side.synchronize()
        assert torch.equal(R, R_ref)


def test_static_scratch_rejects_meshes_beyond_its_capacity():
    pkg = _pkg()
    m = synth.jittered_grid(200, 200, 10.0, 10.0, seed=1)         # 40,000 vertices in FP64
    mesh = pkg.Mesh(m)
    U = torch.from_numpy(synth.uniform_state(m)).cuda()
    R = torch.empty_like(U)
    with pytest.raises(pkg.HfdError) as e:
        mesh.residual_static(mesh.import_state(U), R)
    assert e.value.status == 1
    assert "scratch" in str(e.value)
