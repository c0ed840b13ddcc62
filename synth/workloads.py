"""Composite synthetic workloads.

batched_vortices: many independent isentropic-vortex instances of uneven size, the batched
workload (256 meshes; vertex counts log-uniform in [2e3, 6.4e4]; aspect ratio a ~ U(1, 4);
domain [0, 10a] x [0, 10] with n_x = round(sqrt(V a)), n_y = round(sqrt(V / a)); vortex
strength beta ~ U(2, 5) centred in the domain; mean flow (1, 1)).  Draws, in order from numpy's
PCG64(seed): log V, a, beta for all instances; each mesh then uses seed*100003 + k.
"""
import numpy as np

from .meshes import jittered_grid
from .states import isentropic_vortex


def batched_vortices(n=256, seed=4, vmin=2e3, vmax=6.4e4):
    rng = np.random.Generator(np.random.PCG64(seed))
    logv = rng.uniform(np.log(vmin), np.log(vmax), n)
    aspect = rng.uniform(1.0, 4.0, n)
    beta = rng.uniform(2.0, 5.0, n)
    out = []
    for k in range(n):
        V, a = float(np.exp(logv[k])), float(aspect[k])
        nx, ny = max(8, int(round(np.sqrt(V * a)))), max(8, int(round(np.sqrt(V / a))))
        Lx, Ly = 10.0 * a, 10.0
        m = jittered_grid(nx, ny, Lx, Ly, seed=seed * 100003 + k)
        U = isentropic_vortex(m, beta=float(beta[k]), center=(0.5 * Lx, 0.5 * Ly))
        out.append({"mesh": m, "U": U, "beta": float(beta[k]), "aspect": a})
    return out
