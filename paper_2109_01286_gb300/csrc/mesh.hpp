// Internal definition of the device mesh handle of the C ABI (api.cu, noalloc.cu).
#pragma once
#include <cuda_runtime.h>

#include <map>
#include <utility>
#include <vector>

#include "hfd.h"
#include "kernels.hpp"

struct GraphEntry {
  cudaGraphExec_t exec = nullptr;
};

struct hfd_mesh {
  hfd_options opts{};
  hfd::DevMesh dm;
  hfd::Phys ph{};
  int lanes = 8;
  std::vector<int32_t> perm;            // internal -> input
  int32_t* dperm = nullptr;             // device copy of perm
  double* U1 = nullptr;                 // stage buffers 12 x V
  double* U2 = nullptr;
  double* Uin = nullptr;                // end-to-end staging (input order)
  double* Uint = nullptr;               // end-to-end staging (internal order)
  cudaStream_t cap = nullptr;           // private stream used for graph capture
  std::map<std::pair<const double*, double>, GraphEntry> graphs;
  hfd_mesh_stats stats{};
  std::vector<void*> allocs;
  int device = 0;
};

