// Host preprocessing result and device arrays of the three-dimensional extension.
#pragma once
#include <cstdint>
#include <vector>

#include "hfd3d.h"

namespace hfd {

// Everything geometry-only of a periodic tetrahedral mesh (host, FP64).  Edge arrays are
// edge-major (the layout of hfd3_prep_get); the device copies are structure-of-arrays.
struct Prep3 {
  int V = 0, E = 0;
  double L[3] = {0, 0, 0};
  std::vector<double> x, y, z;
  std::vector<int32_t> edges;                 // 2E (tail < head), sorted
  std::vector<int32_t> nbr_ptr, nbr_idx;      // sorted neighbour lists
  std::vector<int32_t> sten;                  // 6E
  std::vector<double> frame;                  // 9E: n, t1, t2
  std::vector<double> w5;                     // 40E: side, node, (v, x, y, z)
  std::vector<double> w3;                     // 18E: side, candidate, 3
  std::vector<int32_t> rank;                  // 2E
  std::vector<int32_t> vptr, vidx, eptr, eidx;
  std::vector<double> cv;                     // 12 per vertex entry: row (d0, dx, dy, dz) x flux
  std::vector<double> ce;                     // 4 per edge entry
  int64_t deficient = 0;
  int64_t micros = 0;
  void disp(int a, int b, double* d) const;   // minimum-image vector from vertex a to b
};

// Builds the preprocessing; HFD_OK or an error status with hfd_last_error set.
hfd_status build_prep3(const hfd3_mesh_desc* d, const hfd3_options* o, Prep3* P);

// Device arrays of a 3D mesh.
struct DevMesh3 {
  int V = 0, E = 0;
  int lanes = 4;                // threads per vertex in the divergence gather (1, 2, 4)
  int32_t* sten = nullptr;      // 6 x E (SoA)
  double* frame = nullptr;      // 9 x E (SoA)
  double* w5 = nullptr;         // 40 x E (SoA)
  double* w3 = nullptr;         // 18 x E (SoA)
  int32_t *vptr = nullptr, *vidx = nullptr, *eptr = nullptr, *eidx = nullptr;
  double* cv = nullptr;         // 12 per vertex entry (entry-major)
  double* ce = nullptr;         // 4 per edge entry (entry-major)
  double* Ua = nullptr;         // 20 per vertex (vertex-major copy of the state)
  double* FGK = nullptr;        // 15 per vertex: F, G, K
  double* h = nullptr;          // 5 per edge
  double* U1 = nullptr;         // stage scratch states (20 x V)
  double* U2 = nullptr;
  unsigned* err = nullptr;      // error word
};

struct Phys3 {
  double gamma, g1, eps, sens_lo, sens_hi, harten, half_inv_harten;
  float epsf, sens_lof, sens_hif;   // the sensor's constants rounded once to FP32 (host)
  int force_branch;
};

}  // namespace hfd
