// Internal definition of the device mesh handle of the C ABI (api.cu, noalloc.cu).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "hfd.h"
#include "kernels.hpp"

struct GraphEntry {
  cudaGraphExec_t exec = nullptr;
};

namespace hfd {
// NVTX range over a host scope (an API call, a Runge-Kutta stage): it shows in Nsight timelines
// and costs a few nanoseconds when no tool is attached.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
}  // namespace hfd

struct hfd_mesh {
  hfd_options opts{};
  hfd::DevMesh dm;
  hfd::Phys ph{};
  int lanes = 4;                        // lanes per vertex in the divergence kernel (1, 2, 4, 8)
  int persistent = 0;                   // 1: one cooperative launch per RK stage
  int grid = 0;                         // blocks of the persistent launch (0: all resident)
  std::vector<int32_t> perm;            // internal -> input
  std::vector<int32_t> fperm;           // internal flux edge -> the prep's flux-edge index
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
  // adjoint (built on the first hfd_adjoint call): transposed divergence / stencil lists,
  // per-edge node sensitivities [Ef][72], two adjoint stage buffers 12 x V, the list of edges
  // with a 3-node or re-decided component and its length
  int32_t *adj_tv_ptr = nullptr, *adj_tv_row = nullptr, *adj_tv_pos = nullptr;
  int32_t *adj_te_ptr = nullptr, *adj_te_row = nullptr, *adj_te_pos = nullptr;
  int32_t *adj_ts_ptr = nullptr, *adj_ts_ent = nullptr;
  double *adj_Ge = nullptr, *adj_B1 = nullptr, *adj_B2 = nullptr;
  int32_t *adj_list = nullptr, *adj_count = nullptr;
  // transpose of the transmissive ghost refresh (meshes with ghosts): unique donors, the CSR of
  // each donor's ghosts in ascending order with their flags; scratch for the step input with
  // refreshed ghosts and for the transposed lambda_{n+1}
  int32_t adj_ndonor = 0;
  int32_t *adj_gt_donor = nullptr, *adj_gt_ptr = nullptr, *adj_gt_ghost = nullptr,
          *adj_gt_flags = nullptr;
  double *adj_U0 = nullptr, *adj_L = nullptr;
};

// A device block of the mesh: from the caller's allocator (hfd_options.dev_alloc) if there is
// one, else cudaMalloc; recorded for hfd_mesh_destroy.  Blocks must be 256-byte aligned.
inline cudaError_t mesh_malloc(hfd_mesh* m, void** p, size_t bytes) {
  *p = nullptr;
  if (m->opts.dev_alloc) {
    void* q = m->opts.dev_alloc(bytes, m->opts.alloc_ctx);
    if (!q) return cudaErrorMemoryAllocation;
    if (reinterpret_cast<uintptr_t>(q) % 256 != 0) {
      m->opts.dev_free(q, m->opts.alloc_ctx);
      return cudaErrorMisalignedAddress;
    }
    *p = q;
  } else {
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) return e;
  }
  m->allocs.push_back(*p);
  m->stats.device_bytes += (int64_t)bytes;
  return cudaSuccess;
}

// Releases every block of the mesh (the current device must be the mesh's).
inline void mesh_free_all(hfd_mesh* m) {
  if (m->opts.dev_alloc) {
    cudaDeviceSynchronize();     // no kernel may still use a block the allocator reuses
    for (void* p : m->allocs) m->opts.dev_free(p, m->opts.alloc_ctx);
  } else {
    for (void* p : m->allocs) cudaFree(p);
  }
  m->allocs.clear();
}
