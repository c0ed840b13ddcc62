"""Seeded synthetic inputs shared by the CUDA path's tests/bench and by the oracle.

This package holds no arithmetic of the Hermite finite-difference method itself: only
triangle meshes (jittered, randomly split structured grids standing in for the paper's
Delaunay meshes, Sec. 3) and the initial/exact states of the paper's test problems
(isentropic vortex, Sec. 3.1; Couette flow, Sec. 3.2; circular Sod and its
embedded-circle mesh, Sec. 3.3) and of the synthetic workloads (four-quadrant Riemann
problem, planar Sod, Taylor-Green vortex).
"""
from .meshes import (jittered_grid, jittered_box_with_ghosts, couette_channel,
                     embedded_circle_box, mesh_summary, vertex_areas)
from .states import (GAMMA, isentropic_vortex, four_quadrant, planar_sod, taylor_green,
                     uniform_state, prim_to_cons, couette, circular_sod)
from .workloads import batched_vortices

__all__ = ["jittered_grid", "jittered_box_with_ghosts", "couette_channel", "embedded_circle_box", "mesh_summary", "vertex_areas", "GAMMA",
           "isentropic_vortex", "four_quadrant", "planar_sod", "taylor_green",
           "uniform_state", "prim_to_cons", "couette", "circular_sod", "batched_vortices"]
