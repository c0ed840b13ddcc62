// Launchers of the 3D extension's kernels (kernels3d.cu).
#pragma once
#include <cuda_runtime.h>

#include "mesh3.hpp"

namespace hfd {

// Vertex-major copy of U (20 x V) into m.Ua and the flux vectors F, G, K into m.FGK.
cudaError_t launch3_vertex(const DevMesh3& m, const double* U, const Phys3& ph, cudaStream_t s);
// Edge fluxes h from m.Ua (Alg. 1 in 3D and Roe's flux).
cudaError_t launch3_edge(const DevMesh3& m, const Phys3& ph, cudaStream_t s);
// Divergence gather: mode 0 writes R = -div into out; mode 1 writes b (Us + dt R) + a Un.
cudaError_t launch3_div(const DevMesh3& m, const double* Us, const double* Un, double* out,
                        int mode, double a, double b, double dt, cudaStream_t s);

}  // namespace hfd
