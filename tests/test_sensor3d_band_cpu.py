"""The 3D edge kernel's sensor scheme, emulated on the CPU: the WENO test taken in FP32 on the
five-wave projections of the nodes' differences from the tail state (each difference formed in
FP64 and rounded once), with every decision inside a 1e-3 band around a threshold (or with a
non-finite sum) taken again in FP64.  On smooth, shock and developed 3D states, no FP32 decision
outside the band differs from the FP64 decision of the oracle, and the band holds few sides.
(The kernel's own decisions are checked by the GPU parity tests, which compare against the
all-FP64 oracle with nothing excluded.)"""
import numpy as np
import pytest

from oracle import hfd3d as O
from synth import three_d as T

F = np.float32


def _weno_t(u, eps):
    u0, u1, u2, u3, u4 = u
    e1, f1 = u0 - F(2) * u1 + u2, u0 - F(4) * u1 + F(3) * u2
    e2, f2 = u1 - F(2) * u2 + u3, u1 - u3
    e3, f3 = u2 - F(2) * u3 + u4, F(3) * u2 - F(4) * u3 + u4
    s1 = F(eps) + (F(13.0 / 12.0) * (e1 * e1) + F(0.25) * (f1 * f1))
    s2 = F(eps) + (F(13.0 / 12.0) * (e2 * e2) + F(0.25) * (f2 * f2))
    s3 = F(eps) + (F(13.0 / 12.0) * (e3 * e3) + F(0.25) * (f3 * f3))
    s1, s2, s3 = s1 * s1, s2 * s2, s3 * s3
    t0 = F(0.0625) * (s2 * s3)
    return t0, t0 + F(0.625) * (s1 * s3) + F(0.3125) * (s1 * s2)


@pytest.fixture(scope="module")
def box8():
    m = T.periodic_tet_box(8, 8, 8, 10.0, 10.0, 10.0, seed=3)
    return m, O.prepare(m)


@pytest.mark.parametrize("state", ["vortex", "wave", "sod", "sod_after_2_steps"])
def test_fp32_sensor_with_fp64_band_decides_as_fp64(box8, state):
    m, P = box8
    opts = P.opts
    if state == "vortex":
        U = T.vortex_tube(m)
    elif state == "wave":
        U = T.density_wave(m, amp=0.1)
    else:
        U = T.planar_sod3(m)
        if state == "sod_after_2_steps":
            dt = 0.5 * O.cfl_dt(m, P, U)
            U = O.step(m, P, O.step(m, P, U, dt), dt)
    W = U[:, P.stencil]
    wi, wj = W[0:5, :, 2], W[0:5, :, 3]
    vel, H, c = O.roe_average(wi, wj, opts.gamma)
    L, R = O.eigenvectors(vel, H, c, P.normal, P.t1, P.t2, opts.gamma)
    C64 = np.einsum("eij,jek->eik", L, W[0:5])
    C32 = np.einsum("eij,jek->eik", L.astype(F), (W[0:5] - wi[:, :, None]).astype(F))
    differ = band = total = 0
    for order in ([0, 1, 2, 3, 4], [5, 4, 3, 2, 1]):
        o1, _, _ = O.weno_weights(*[C64[:, :, k] for k in order], opts.weno_eps)
        smooth64 = (o1 > opts.sens_lo) & (o1 < opts.sens_hi)
        with np.errstate(over="ignore", invalid="ignore"):
            t0, S = _weno_t([C32[:, :, k] for k in order], opts.weno_eps)
            mlo, mhi = t0 - F(opts.sens_lo) * S, F(opts.sens_hi) * S - t0
            clear = np.isfinite(S) & (np.abs(mlo) > F(1e-3) * S) & (np.abs(mhi) > F(1e-3) * S)
        differ += int(np.sum(clear & (((mlo > 0) & (mhi > 0)) != smooth64)))
        band += int(np.sum(~clear))
        total += smooth64.size
    assert differ == 0
    assert band < 0.02 * total
