// hfd_residual_static: the right-hand side R(U) with its per-call scratch in a fixed device
// array compiled into the library, so the call itself allocates no device memory.
//
// Who needs it: an application that reserves all device memory up front for its own pool and
// lets libraries use only what they were given (fixed memory budgets, long-running services),
// and code that must not call cudaMalloc / cudaFree while other work runs on the device, since
// those calls can synchronise the whole device.  Such a caller creates its meshes once at start
// up and then evaluates residuals without any further allocation.
//
// The scratch -- the AoS copy of the state, the vertex fluxes and the edge fluxes -- lives in
// g_static_scratch below, HFD_STATIC_SCRATCH_BYTES per device.  Every GPU that loads the
// library holds that array until the process exits.  All calls on a device share the one
// array: calls whose work overlaps on the GPU (different streams, or different host threads)
// race on it and must be serialised by the caller.  Each call fully overwrites the parts of
// the array it reads before reading them, so nothing has to start at zero and no contents of an
// earlier call leak into a later one.
#include <cuda_runtime.h>

#include <cstdio>

#include "kernels.hpp"
#include "mesh.hpp"
#include "prep.hpp"

#define HFD_STATIC_SCRATCH_BYTES (8u << 20)

static __device__ __align__(256) unsigned char g_static_scratch[HFD_STATIC_SCRATCH_BYTES];

namespace {

// In host code g_static_scratch names a host-side stand-in, not device memory: the kernels
// must be given the device address, looked up with the mesh's device current.  The lookup is
// repeated on every call (it allocates nothing and costs a host-side table search once the
// library's device code is loaded): a cached address would go stale if the device's context
// were destroyed and created again (cudaDeviceReset), since the array may then live elsewhere.
hfd_status static_scratch_address(void** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
  if (e != cudaSuccess || !p) {
    hfd::set_error("hfd_residual_static: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    return HFD_ERR_CUDA;
  }
  *out = p;
  return HFD_OK;
}

size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

extern "C" hfd_status hfd_residual_static(hfd_mesh* m, double* U, double* R, void* stream) {
  if (!m || !U || !R || U == R) {
    hfd::set_error("hfd_residual_static: invalid argument");
    return HFD_ERR_ARG;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != m->device) {
    hfd::set_error("hfd_residual_static: the mesh lives on device %d; make it current", m->device);
    return HFD_ERR_ARG;
  }
  const hfd::DevMesh& src = m->dm;
  const size_t T = src.precision == 0 ? sizeof(double) : sizeof(float);
  const size_t V = (size_t)src.V, Ef = (size_t)src.Ef;
  const size_t b_ua = round256(V * 12 * T), b_fg = round256(V * 8 * T);
  const size_t b_fgv = src.viscous ? round256(V * 8 * T) : 0, b_h = round256(Ef * 4 * T);
  const size_t need = b_ua + b_fg + b_fgv + b_h;
  if (need > HFD_STATIC_SCRATCH_BYTES) {
    hfd::set_error("hfd_residual_static: mesh needs %zu bytes of scratch (%zu vertices, %zu flux "
                   "edges), above the fixed %u-byte array; use hfd_residual",
                   need, V, Ef, (unsigned)HFD_STATIC_SCRATCH_BYTES);
    return HFD_ERR_ARG;
  }
  void* base = nullptr;
  hfd_status st = static_scratch_address(&base);
  if (st != HFD_OK) return st;
  hfd::DevMesh d = src;                          // same streams, scratch redirected
  unsigned char* p = static_cast<unsigned char*>(base);
  d.Ua = p;
  d.FG = p + b_ua;
  d.FGv = src.viscous ? p + b_ua + b_fg : nullptr;
  d.h = p + b_ua + b_fg + b_fgv;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = hfd::launch_ghost(d, U, U, s);
  if (e == cudaSuccess) e = hfd::launch_vertex(d, U, m->ph, s);
  if (e == cudaSuccess) e = hfd::launch_edge(d, m->ph, s);
  if (e == cudaSuccess)
    e = hfd::launch_div(d, U, U, R, hfd::DIV_RESIDUAL, 0.0, 1.0, 1.0, m->ph, m->lanes, s);
  if (e == cudaSuccess && d.V > d.A)
    e = cudaMemset2DAsync(R + d.A, V * sizeof(double), 0, (V - (size_t)d.A) * sizeof(double), 12, s);
  if (e != cudaSuccess) {
    hfd::set_error("hfd_residual_static: %s", cudaGetErrorString(e));
    return HFD_ERR_CUDA;
  }
  return HFD_OK;
}
