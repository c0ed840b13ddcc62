// C ABI of the three-dimensional extension (include/hfd3d.h): mesh creation (host
// preprocessing in prep3.cpp, upload), residual, SSP-RK3 steps, preprocessing access.
#include <cuda_runtime.h>

#include <cstring>
#include <string>
#include <vector>

#include "hfd3d.h"
#include "kernels3d.hpp"
#include "prep.hpp"

struct hfd3_mesh {
  hfd::Prep3 P;
  hfd::DevMesh3 d;
  hfd::Phys3 ph;
  hfd3_options opts;
  std::vector<void*> allocs;
};

namespace {

using hfd::set_error;

#define CK3(call)                                                            \
  do {                                                                       \
    cudaError_t e_ = (call);                                                 \
    if (e_ != cudaSuccess) {                                                 \
      set_error("%s: %s", __func__, cudaGetErrorString(e_));                 \
      return HFD_ERR_CUDA;                                                   \
    }                                                                        \
  } while (0)

hfd_status dalloc(hfd3_mesh* m, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    set_error("hfd3_mesh_create: cudaMalloc of %zu bytes: %s", bytes, cudaGetErrorString(e));
    return HFD_ERR_CUDA;
  }
  m->allocs.push_back(*p);
  return HFD_OK;
}

// edge-major host array (k values per edge) -> k x E structure-of-arrays
template <typename T>
std::vector<T> to_soa(const std::vector<T>& a, int E, int k) {
  std::vector<T> o((size_t)k * E);
  for (int e = 0; e < E; ++e)
    for (int j = 0; j < k; ++j) o[(size_t)j * E + e] = a[(size_t)k * e + j];
  return o;
}

template <typename T>
hfd_status put(const std::vector<T>& h, T* dptr) {
  if (h.empty()) return HFD_OK;
  cudaError_t e = cudaMemcpy(dptr, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    set_error("hfd3: upload: %s", cudaGetErrorString(e));
    return HFD_ERR_CUDA;
  }
  return HFD_OK;
}

#define TRY3(x)                          \
  do {                                   \
    hfd_status s_ = (x);                 \
    if (s_ != HFD_OK) return s_;         \
  } while (0)

hfd_status upload_edges(hfd3_mesh* m) {
  const int E = m->P.E;
  TRY3(put(to_soa(m->P.sten, E, 6), m->d.sten));
  TRY3(put(to_soa(m->P.frame, E, 9), m->d.frame));
  TRY3(put(to_soa(m->P.w5, E, 40), m->d.w5));
  TRY3(put(to_soa(m->P.w3, E, 18), m->d.w3));
  return HFD_OK;
}

hfd_status create(const hfd3_mesh_desc* desc, const hfd3_options* o, hfd3_mesh* m) {
  TRY3(hfd::build_prep3(desc, o, &m->P));
  const hfd::Prep3& P = m->P;
  hfd::DevMesh3& d = m->d;
  d.V = P.V;
  d.E = P.E;
  if (o->host_only) return HFD_OK;           // host preprocessing only: nothing on the device
  const size_t V = P.V, E = P.E;
  TRY3(dalloc(m, (void**)&d.sten, 6 * E * sizeof(int32_t)));
  TRY3(dalloc(m, (void**)&d.frame, 9 * E * sizeof(double)));
  TRY3(dalloc(m, (void**)&d.w5, 40 * E * sizeof(double)));
  TRY3(dalloc(m, (void**)&d.w3, 18 * E * sizeof(double)));
  TRY3(dalloc(m, (void**)&d.vptr, (V + 1) * sizeof(int32_t)));
  TRY3(dalloc(m, (void**)&d.eptr, (V + 1) * sizeof(int32_t)));
  TRY3(dalloc(m, (void**)&d.vidx, P.vidx.size() * sizeof(int32_t)));
  TRY3(dalloc(m, (void**)&d.eidx, P.eidx.size() * sizeof(int32_t)));
  TRY3(dalloc(m, (void**)&d.cv, P.cv.size() * sizeof(double)));
  TRY3(dalloc(m, (void**)&d.ce, P.ce.size() * sizeof(double)));
  TRY3(dalloc(m, (void**)&d.Ua, 20 * V * sizeof(double)));
  TRY3(dalloc(m, (void**)&d.FGK, 16 * V * sizeof(double)));
  TRY3(dalloc(m, (void**)&d.h, 8 * E * sizeof(double)));
  TRY3(dalloc(m, (void**)&d.U1, 20 * V * sizeof(double)));
  TRY3(dalloc(m, (void**)&d.U2, 20 * V * sizeof(double)));
  TRY3(dalloc(m, (void**)&d.err, sizeof(unsigned)));
  CK3(cudaMemset(d.err, 0, sizeof(unsigned)));
  TRY3(upload_edges(m));
  TRY3(put(P.vptr, d.vptr));
  TRY3(put(P.eptr, d.eptr));
  TRY3(put(P.vidx, d.vidx));
  TRY3(put(P.eidx, d.eidx));
  TRY3(put(P.cv, d.cv));
  TRY3(put(P.ce, d.ce));
  m->ph.gamma = o->gamma;
  m->ph.g1 = o->gamma - 1.0;
  m->ph.eps = o->weno_eps;
  m->ph.sens_lo = o->sens_lo;
  m->ph.sens_hi = o->sens_hi;
  m->ph.harten = o->harten;
  m->ph.half_inv_harten = 0.5 / o->harten;
  m->ph.epsf = (float)o->weno_eps;
  m->ph.sens_lof = (float)o->sens_lo;
  m->ph.sens_hif = (float)o->sens_hi;
  m->ph.force_branch = o->force_branch;
  return HFD_OK;
}

// One named host array: pointer, element count, element size, writable
struct Named {
  void* p;
  int64_t n;
  size_t elt;
  bool writable;
};

Named lookup(const hfd3_mesh* cm, const char* name) {
  hfd3_mesh* m = const_cast<hfd3_mesh*>(cm);
  hfd::Prep3& P = m->P;
  auto I = [](std::vector<int32_t>& v, bool w) { return Named{v.data(), (int64_t)v.size(), 4, w}; };
  auto D = [](std::vector<double>& v, bool w) { return Named{v.data(), (int64_t)v.size(), 8, w}; };
  if (!name) return {nullptr, -1, 0, false};
  const std::string s(name);
  if (s == "edges") return I(P.edges, false);
  if (s == "sten") return I(P.sten, true);
  if (s == "frame") return D(P.frame, true);
  if (s == "w5") return D(P.w5, true);
  if (s == "w3") return D(P.w3, true);
  if (s == "rank") return I(P.rank, false);
  if (s == "vptr") return I(P.vptr, false);
  if (s == "vidx") return I(P.vidx, false);
  if (s == "eptr") return I(P.eptr, false);
  if (s == "eidx") return I(P.eidx, false);
  if (s == "cv") return D(P.cv, true);
  if (s == "ce") return D(P.ce, true);
  return {nullptr, -1, 0, false};
}

hfd_status stage(hfd3_mesh* m, const double* Uin, const double* Us, const double* Un, double* out,
                 double a, double b, double dt, cudaStream_t s, cudaEvent_t* ev) {
  if (ev) CK3(cudaEventRecord(ev[0], s));
  CK3(hfd::launch3_vertex(m->d, Uin, m->ph, s));
  if (ev) CK3(cudaEventRecord(ev[1], s));
  CK3(hfd::launch3_edge(m->d, m->ph, s));
  if (ev) CK3(cudaEventRecord(ev[2], s));
  CK3(hfd::launch3_div(m->d, Us, Un, out, 1, a, b, dt, s));
  if (ev) CK3(cudaEventRecord(ev[3], s));
  return HFD_OK;
}

}  // namespace

extern "C" {

void hfd3_default_options(hfd3_options* o) {
  if (!o) return;
  o->gamma = 1.4;
  o->weno_eps = 1e-2;
  o->sens_lo = 0.01;
  o->sens_hi = 0.79;
  o->harten = 0.1;
  o->sv_rtol = 1e-13;
  o->div_cond_min = 1e-12;
  o->force_branch = 0;
  o->threads = 0;
  o->host_only = 0;
}

hfd_status hfd3_mesh_create(const hfd3_mesh_desc* desc, const hfd3_options* opts, hfd3_mesh** out) {
  if (!out) {
    set_error("hfd3_mesh_create: null output");
    return HFD_ERR_ARG;
  }
  *out = nullptr;
  hfd3_options o;
  hfd3_default_options(&o);
  if (opts) o = *opts;
  if (!(o.gamma > 1.0) || !(o.harten > 0.0) || o.force_branch < 0 || o.force_branch > 2 ||
      (o.host_only != 0 && o.host_only != 1)) {
    set_error("hfd3_mesh_create: invalid options");
    return HFD_ERR_ARG;
  }
  hfd3_mesh* m = new hfd3_mesh();
  m->opts = o;
  hfd_status st = create(desc, &o, m);
  if (st != HFD_OK) {
    hfd3_mesh_destroy(m);
    return st;
  }
  *out = m;
  return HFD_OK;
}

void hfd3_mesh_destroy(hfd3_mesh* m) {
  if (!m) return;
  for (void* p : m->allocs) cudaFree(p);
  delete m;
}

hfd_status hfd3_mesh_info(const hfd3_mesh* m, int64_t info[6]) {
  if (!m || !info) {
    set_error("hfd3_mesh_info: invalid argument");
    return HFD_ERR_ARG;
  }
  info[0] = m->P.V;
  info[1] = m->P.E;
  info[2] = (int64_t)m->P.vidx.size();
  info[3] = (int64_t)m->P.eidx.size();
  info[4] = m->P.deficient;
  info[5] = m->P.micros;
  return HFD_OK;
}

int64_t hfd3_prep_size(const hfd3_mesh* m, const char* name) {
  if (!m) return -1;
  return lookup(m, name).n;
}

hfd_status hfd3_prep_get(const hfd3_mesh* m, const char* name, void* dst, int64_t count) {
  if (!m || !dst) {
    set_error("hfd3_prep_get: invalid argument");
    return HFD_ERR_ARG;
  }
  Named a = lookup(m, name);
  if (a.n < 0 || count != a.n) {
    set_error("hfd3_prep_get: unknown name or wrong count for '%s'", name ? name : "(null)");
    return HFD_ERR_ARG;
  }
  std::memcpy(dst, a.p, (size_t)a.n * a.elt);
  return HFD_OK;
}

hfd_status hfd3_prep_set(hfd3_mesh* m, const char* name, const void* src, int64_t count) {
  if (!m || !src) {
    set_error("hfd3_prep_set: invalid argument");
    return HFD_ERR_ARG;
  }
  Named a = lookup(m, name);
  if (a.n < 0 || !a.writable || count != a.n) {
    set_error("hfd3_prep_set: unknown or read-only name, or wrong count, for '%s'",
              name ? name : "(null)");
    return HFD_ERR_ARG;
  }
  if (std::string(name) == "sten") {
    const int32_t* s = static_cast<const int32_t*>(src);
    for (int64_t i = 0; i < count; ++i)
      if (s[i] < 0 || s[i] >= m->P.V) {
        set_error("hfd3_prep_set: stencil id out of range");
        return HFD_ERR_ARG;
      }
  }
  std::memcpy(a.p, src, (size_t)a.n * a.elt);
  if (!m->d.err) return HFD_OK;               // host-only mesh: no device copy to refresh
  const std::string s(name);
  if (s == "cv") return put(m->P.cv, m->d.cv);
  if (s == "ce") return put(m->P.ce, m->d.ce);
  return upload_edges(m);
}

hfd_status hfd3_residual(hfd3_mesh* m, const double* U, double* R, void* stream) {
  if (!m || !U || !R || U == R) {
    set_error("hfd3_residual: invalid argument");
    return HFD_ERR_ARG;
  }
  if (!m->d.err) {
    set_error("hfd3_residual: the mesh was built host-only");
    return HFD_ERR_UNSUPPORTED;
  }
  cudaStream_t s = (cudaStream_t)stream;
  CK3(hfd::launch3_vertex(m->d, U, m->ph, s));
  CK3(hfd::launch3_edge(m->d, m->ph, s));
  CK3(hfd::launch3_div(m->d, nullptr, nullptr, R, 0, 0.0, 1.0, 0.0, s));
  return HFD_OK;
}

static hfd_status steps_impl(hfd3_mesh* m, double* U, double dt, int32_t nsteps, cudaStream_t s,
                             cudaEvent_t* ev, double* ms) {
  hfd::DevMesh3& d = m->d;
  for (int n = 0; n < nsteps; ++n) {
    // SSP-RK3: U1 = U + dt L(U); U2 = 3/4 U + 1/4 (U1 + dt L(U1)); U = 1/3 U + 2/3 (U2 + dt L(U2))
    const double a[3] = {0.0, 0.75, 1.0 / 3.0}, b[3] = {1.0, 0.25, 2.0 / 3.0};
    const double* in[3] = {U, d.U1, d.U2};
    double* outp[3] = {d.U1, d.U2, U};
    for (int k = 0; k < 3; ++k) {
      TRY3(stage(m, in[k], in[k], k == 0 ? nullptr : U, outp[k], a[k], b[k], dt, s, ev));
      if (ev) {
        CK3(cudaEventSynchronize(ev[3]));
        for (int j = 0; j < 3; ++j) {
          float t = 0.f;
          CK3(cudaEventElapsedTime(&t, ev[j], ev[j + 1]));
          ms[j] += t;
        }
      }
    }
  }
  return HFD_OK;
}

hfd_status hfd3_steps(hfd3_mesh* m, double* U, double dt, int32_t nsteps, void* stream) {
  if (!m || !U || !(dt > 0.0) || nsteps < 0) {
    set_error("hfd3_steps: invalid argument");
    return HFD_ERR_ARG;
  }
  if (!m->d.err) {
    set_error("hfd3_steps: the mesh was built host-only");
    return HFD_ERR_UNSUPPORTED;
  }
  return steps_impl(m, U, dt, nsteps, (cudaStream_t)stream, nullptr, nullptr);
}

hfd_status hfd3_steps_profiled(hfd3_mesh* m, double* U, double dt, int32_t nsteps, double ms[3],
                               void* stream) {
  if (!m || !U || !ms || !(dt > 0.0) || nsteps < 0) {
    set_error("hfd3_steps_profiled: invalid argument");
    return HFD_ERR_ARG;
  }
  if (!m->d.err) {
    set_error("hfd3_steps_profiled: the mesh was built host-only");
    return HFD_ERR_UNSUPPORTED;
  }
  ms[0] = ms[1] = ms[2] = 0.0;
  cudaEvent_t ev[4];
  for (int i = 0; i < 4; ++i) CK3(cudaEventCreate(&ev[i]));
  hfd_status st = steps_impl(m, U, dt, nsteps, (cudaStream_t)stream, ev, ms);
  for (int i = 0; i < 4; ++i) cudaEventDestroy(ev[i]);
  return st;
}

hfd_status hfd3_mesh_set_lanes(hfd3_mesh* m, int32_t lanes) {
  if (!m || (lanes != 1 && lanes != 2 && lanes != 4)) {
    set_error("hfd3_mesh_set_lanes: lanes must be 1, 2 or 4");
    return HFD_ERR_ARG;
  }
  m->d.lanes = lanes;
  return HFD_OK;
}

hfd_status hfd3_check(hfd3_mesh* m) {
  if (!m) {
    set_error("hfd3_check: null mesh");
    return HFD_ERR_ARG;
  }
  if (!m->d.err) return HFD_OK;               // host-only mesh: nothing ran
  CK3(cudaDeviceSynchronize());
  unsigned w = 0;
  CK3(cudaMemcpy(&w, m->d.err, sizeof w, cudaMemcpyDeviceToHost));
  CK3(cudaMemset(m->d.err, 0, sizeof w));
  if (w & 4u) {
    set_error("hfd3_check: a gathered index was out of range");
    return HFD_ERR_MESH;
  }
  if (w & 1u) {
    set_error("hfd3_check: non-finite value in a residual or stage");
    return HFD_ERR_NONFINITE;
  }
  if (w & 2u) {
    set_error("hfd3_check: non-positive density after a stage");
    return HFD_ERR_POSITIVITY;
  }
  return HFD_OK;
}

}  // extern "C"
