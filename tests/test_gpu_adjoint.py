"""GPU tests of the discrete adjoint (hfd_adjoint) and its torch.autograd wrapper."""
import numpy as np
import pytest

import oracle
import synth
from oracle import adjoint as ADJ
from gpu_helpers import inject_oracle_coefficients

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2109_01286_gb300 as pkg
    return pkg


@pytest.mark.parametrize("conservative,flux", [(False, "roe"), (True, "roe"), (False, "rusanov")])
def test_adjoint_step_matches_oracle_adjoint_20x20(conservative, flux):
    """The GPU adjoint of one step against the oracle's adjoint on a 20 x 20 vortex mesh, with
    the oracle's coefficients in both (kernel parity); also for the conservative variant, whose
    coefficients and flux directions the same reverse kernels take, and for Rusanov's flux."""
    pkg = _pkg()
    m = synth.jittered_grid(20, 20, 10.0, 10.0, seed=5)
    U = synth.isentropic_vortex(m)
    opts = oracle.Options(conservative=conservative, flux=flux)
    P = oracle.prepare(m, opts)
    dt = oracle.cfl_dt(m, P, U)
    lam = np.random.default_rng(0).standard_normal(U.shape)
    ref = ADJ.step_vjp(m, P, U, dt, lam, opts)
    prep = pkg.Prep(m, conservative=conservative, flux=flux)
    inject_oracle_coefficients(prep, P, len(m["x"]))
    mesh = prep.upload()
    Ui = mesh.import_state(torch.from_numpy(U).cuda())
    li = mesh.import_state(torch.from_numpy(lam).cuda())
    out = mesh.export_state(mesh.adjoint(Ui, li, dt=dt)).cpu().numpy()
    err = np.linalg.norm(out - ref) / np.linalg.norm(ref)
    assert err < 1e-11, err


@pytest.mark.parametrize("kind", ["transmissive", "walls", "delaunay"])
def test_adjoint_step_with_ghost_layers_matches_oracle_adjoint(kind):
    """Meshes with ghost layers: transmissive ghosts on a box (5 layers), and the fixed wall
    bands of the channel (donor -1, 6 layers), each with a smooth inviscid state.  The GPU
    adjoint of one step against the oracle's (kernel parity): the ghost refresh enters
    transposed on both sides.  Transmissive ghost columns of lam_n are zero; band columns carry
    their sensitivity."""
    pkg = _pkg()
    if kind == "transmissive":
        m = synth.jittered_box_with_ghosts(16, 16, (0.0, 1.0), (0.0, 1.0), 5, seed=5)
        U = synth.isentropic_vortex(m, beta=2.0, center=(0.5, 0.5), mean=(1.0, 0.5))
    elif kind == "walls":
        m = synth.couette_channel(16, 17, 6, seed=7)
        U = synth.isentropic_vortex(m, beta=2.0, center=(0.0, 0.0), mean=(0.5, 0.0))
    else:                                    # the embedded-circle Delaunay mesh, 5 ghost layers
        m = synth.embedded_circle_box(16, seed=8)
        U = synth.isentropic_vortex(m, beta=1.0, center=(0.0, 0.0), mean=(0.5, 0.3))
    P = oracle.prepare(m)
    dt = 0.5 * oracle.cfl_dt(m, P, U)
    lam = np.random.default_rng(1).standard_normal(U.shape)
    ref = ADJ.step_vjp(m, P, U, dt, lam)
    prep = pkg.Prep(m)
    inject_oracle_coefficients(prep, P, len(m["x"]))
    mesh = prep.upload()
    U_dev = torch.from_numpy(U).cuda()
    Ui = mesh.import_state(U_dev)
    U_before = Ui.clone()
    li = mesh.import_state(torch.from_numpy(lam).cuda())
    out = mesh.export_state(mesh.adjoint(Ui, li, dt=dt)).cpu().numpy()
    assert torch.equal(Ui, U_before)                 # the input state is not modified
    err = np.linalg.norm(out - ref) / np.linalg.norm(ref)
    assert err < 1e-11, err
    g, dn = m["ghost_ids"], m["ghost_donor"]
    if kind != "walls":
        assert np.all(out[:, g] == 0.0)
    else:
        assert np.all(dn < 0) and np.linalg.norm(out[:, g]) > 0.0


@pytest.mark.parametrize("case", ["taylor_green", "couette_walls"])
def test_adjoint_step_viscous_matches_oracle_adjoint(case):
    """Viscous meshes: the reverse of the vertex viscous fluxes (chain-rule gradients, Stokes
    stresses, Fourier heat flux) and the transposed viscous rows, against the oracle's adjoint
    (complex-step Jacobians) on a periodic Taylor-Green mesh and on the Sec. 3.2 channel with
    its wall bands (kernel parity)."""
    pkg = _pkg()
    if case == "taylor_green":
        m = synth.jittered_grid(16, 16, 2 * np.pi, 2 * np.pi, seed=3)
        U = synth.taylor_green(m)
        kw = dict(viscous=True, mu=0.05, prandtl=0.72, R_gas=1.0 / (1.4 * 0.01))
    else:
        m = synth.couette_channel(16, 17, 6, seed=7)
        U = synth.couette(m)
        kw = dict(viscous=True, mu=0.1, prandtl=100.0, R_gas=0.4 * 10.0 / 1.4)
    opts = oracle.Options(**kw)
    P = oracle.prepare(m, opts)
    dt = 0.5 * oracle.cfl_dt(m, P, U)
    lam = np.random.default_rng(2).standard_normal(U.shape)
    ref = ADJ.step_vjp(m, P, U, dt, lam, opts)
    prep = pkg.Prep(m, **kw)
    inject_oracle_coefficients(prep, P, len(m["x"]))
    mesh = prep.upload()
    Ui = mesh.import_state(torch.from_numpy(U).cuda())
    li = mesh.import_state(torch.from_numpy(lam).cuda())
    out = mesh.export_state(mesh.adjoint(Ui, li, dt=dt)).cpu().numpy()
    err = np.linalg.norm(out - ref) / np.linalg.norm(ref)
    assert err < 1e-11, err


def test_adjoint_rollout_against_central_differences():
    """<grad, delta> from the autograd rollout (checkpointed adjoint) against central finite
    differences of the objective sum_v A_v (rho - rho_ref)^2 (step 1e-6)."""
    pkg = _pkg()
    m = synth.jittered_grid(32, 32, 10.0, 10.0, seed=6)
    U0 = synth.isentropic_vortex(m)
    mesh = pkg.Mesh(m)
    dt = 0.03
    area = torch.from_numpy(oracle.vertex_areas(m)).cuda()
    rho_ref = torch.from_numpy(synth.isentropic_vortex(m, t=10 * dt)[0]).cuda()
    perm = torch.from_numpy(mesh.perm.astype(np.int64)).cuda()
    area_i, rho_ref_i = area[perm], rho_ref[perm]

    def J(Ui):
        UN = pkg.autograd.rollout(Ui, mesh, dt, 10, every=4)
        return torch.sum(area_i * (UN[0] - rho_ref_i) ** 2)

    U0i = mesh.import_state(torch.from_numpy(U0).cuda()).requires_grad_(True)
    val = J(U0i)
    val.backward()
    g = U0i.grad.detach()
    rng = np.random.default_rng(7)
    for _ in range(4):
        d = torch.from_numpy(rng.standard_normal(U0.shape)).cuda()
        d = mesh.import_state(d)
        eps = 1e-6
        with torch.no_grad():
            jp = J((U0i + eps * d).detach()).item()
            jm = J((U0i - eps * d).detach()).item()
        fd = (jp - jm) / (2 * eps)
        ad = torch.sum(g * d).item()
        assert abs(fd - ad) <= 1e-5 * max(abs(fd), 1e-12), (fd, ad)


def test_adjoint_rollout_with_ghost_layers_against_central_differences():
    """The checkpointed rollout on a box with 5 transmissive ghost layers: <grad, delta>
    against central differences of J = sum over physical vertices of A_v (rho - rho_ref)^2.
    Perturbations of the ghost columns change nothing (every step refreshes them), and the
    gradient there is zero."""
    pkg = _pkg()
    m = synth.jittered_box_with_ghosts(24, 24, (0.0, 1.0), (0.0, 1.0), 5, seed=12)
    U0 = synth.isentropic_vortex(m, beta=2.0, center=(0.5, 0.5), mean=(1.0, 0.5))
    mesh = pkg.Mesh(m)
    dt = 0.002
    perm = torch.from_numpy(mesh.perm.astype(np.int64)).cuda()
    area = torch.from_numpy(synth.vertex_areas(m)).cuda()
    area[torch.from_numpy(m["ghost_ids"].astype(np.int64)).cuda()] = 0.0
    rho_ref = torch.from_numpy(synth.isentropic_vortex(m, beta=2.0, center=(0.5, 0.5),
                                                       mean=(1.0, 0.5), t=6 * dt)[0]).cuda()
    area_i, rho_ref_i = area[perm], rho_ref[perm]

    def J(Ui):
        UN = pkg.autograd.rollout(Ui, mesh, dt, 6, every=2)
        return torch.sum(area_i * (UN[0] - rho_ref_i) ** 2)

    U0i = mesh.import_state(torch.from_numpy(U0).cuda()).requires_grad_(True)
    J(U0i).backward()
    g = U0i.grad.detach()
    ghosts_i = torch.isin(perm, torch.from_numpy(m["ghost_ids"].astype(np.int64)).cuda())
    assert torch.all(g[:, ghosts_i] == 0.0)
    rng = np.random.default_rng(8)
    for _ in range(4):
        d = mesh.import_state(torch.from_numpy(rng.standard_normal(U0.shape)).cuda())
        eps = 1e-6
        with torch.no_grad():
            fd = (J((U0i + eps * d).detach()).item() - J((U0i - eps * d).detach()).item()) / (2 * eps)
        ad = torch.sum(g * d).item()
        assert abs(fd - ad) <= 1e-5 * max(abs(fd), 1e-12), (fd, ad)
