"""Plain, slow FP64 CPU oracle of the Hermite finite-difference method (arXiv 2109.01286).

TEST INFRASTRUCTURE ONLY.  Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline and
reference legs of `bench.py` may import it.  The product path (the CUDA library and its Python
binding) never imports, links or calls anything here, and this package shares no code with it:
it has its own topology, stencil assembly, pseudo-inverses (numpy/LAPACK SVD), fluxes and time
stepping.  The only module both sides use is `synth` (seeded meshes and initial states), which
holds none of the method's arithmetic.

Every function cites the part of the paper it follows.  Readings of passages the paper leaves
open are tagged R1..R20 and listed in the repository's design notes.  `hfd3d` is the oracle of
the three-dimensional extension (readings T1..T6).
"""
from .hfd_oracle import (Options, build_topology, edge_stencil, taylor_basis, five_node_weights,
                         three_node_weights, edge_geometry, vertex_stencil, div_rows, visc_rows,
                         prepare, euler_flux, viscous_flux, roe_average, eigenvectors,
                         weno_weights, roe_flux, rusanov_flux, riemann_flux, ghost_fill, residual, ssp_rk3, step, cfl_dt,
                         vertex_areas)
from . import hfd3d

__all__ = ["Options", "build_topology", "edge_stencil", "taylor_basis", "five_node_weights",
           "three_node_weights", "edge_geometry", "vertex_stencil", "div_rows", "visc_rows",
           "prepare", "euler_flux", "viscous_flux", "roe_average", "eigenvectors",
           "weno_weights", "roe_flux", "rusanov_flux", "riemann_flux", "ghost_fill", "residual", "ssp_rk3", "step", "cfl_dt",
           "vertex_areas", "hfd3d"]
