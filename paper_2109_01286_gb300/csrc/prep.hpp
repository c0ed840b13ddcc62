// Internal definitions shared by the host preprocessing (prep.cpp) and the device mesh (api.cu).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "hfd.h"

namespace hfd {

void set_error(const char* fmt, ...);

// Geometry-only data of a mesh, in input numbering (see hfd_prep_* in hfd.h).
struct Prep {
  hfd_options opts;
  // mesh
  int32_t nv = 0;
  std::vector<double> x, y;
  std::vector<int32_t> tri;
  double Lx = 0, Ly = 0;
  int periodic_x = 0, periodic_y = 0;
  std::vector<int32_t> ghost_ids, ghost_donor, ghost_flags;
  std::vector<uint8_t> is_ghost;
  // topology: sorted unique edges (tail < head) and sorted neighbour lists with edge ids
  std::vector<int32_t> edges;                  // 2*E
  std::vector<int32_t> nbr_ptr, nbr_idx, nbr_edge;
  // divergence rows of the active (non-ghost) vertices, ascending input id
  std::vector<int32_t> active;
  std::vector<int32_t> div_vptr, div_vidx, div_eptr, div_eidx, div_degree;
  std::vector<int64_t> div_cptr;               // start of each vertex's 3*(2N+M) block
  std::vector<double> div_coef;
  std::vector<int64_t> visc_cptr;              // start of each vertex's 3*2N block
  std::vector<double> visc_coef;
  std::vector<int32_t> visc_degree;            // degree kept per active vertex (viscous)
  // edges whose flux the divergence reads (ascending edge index) and their interpolation data
  std::vector<int32_t> flux_edges;             // Ef
  std::vector<int32_t> stencil;                // 6*Ef, input ids [i-2 .. i+3]
  std::vector<double> normal;                  // 2*Ef
  std::vector<double> w5;                      // 30*Ef: side L (15) then side R (15)
  std::vector<double> w3;                      // 18*Ef: side, sub-stencil, node
  std::vector<int32_t> rank;                   // 2*Ef
  std::vector<double> lmin;                    // nv: shortest incident edge (time step)
  // conservative variant: dual-face area vectors (2*E, oriented tail -> head) and median-dual
  // cell areas (nv)
  std::vector<double> dual_S, dual_A;
  // batches (hfd_prep_concat): member mesh of each vertex and each member's bounding box
  // (x0, x1, y0, y1) for the space-filling-curve keys; empty / 1 for a single mesh
  std::vector<int32_t> member;
  int32_t nmember = 1;
  std::vector<double> member_box;
  int64_t degree_fallbacks = 0;
  int64_t visc_fallbacks = 0;
  double prep_seconds = 0;

  int64_t nedges() const { return (int64_t)edges.size() / 2; }
  double dispx(int a, int b) const;
  double dispy(int a, int b) const;
};

hfd_status build_prep(const hfd_mesh_desc* d, const hfd_options* o, Prep* p);

}  // namespace hfd

// The opaque handle of the C ABI is the preprocessing object itself.
struct hfd_prep : hfd::Prep {};
