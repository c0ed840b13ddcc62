/* hfd3d.h: C ABI of the three-dimensional extension of the Hermite finite-difference residual
 * and SSP-RK3 step (arXiv 2109.01286 is two-dimensional; Sec. 4 names three dimensions as
 * future work).  The extension carries every step of the 2D method over to tetrahedral meshes:
 * curvilinear 6-node edge stencils (Sec. 2.1), Hermite least squares on 5 nodes with the data
 * w, w_x, w_y, w_z and the complete degree-3 Taylor basis (Sec. 2.2), the characteristic WENO
 * sensor and 3-node candidates of Alg. 1 with five waves, Roe's flux, the two-level
 * least-squares divergence of the three flux vectors with degree-4 polynomials (Sec. 2.3,
 * Eq. (flux_polynomials)) fused with the SSP-RK3 stage update.  Inviscid equations on periodic
 * boxes; FP64 throughout.
 *
 * State: 20 x nv float64 device arrays, row-major by row (row r of vertex v at r*nv + v), in the
 * input vertex order: rows 0-4 w = (rho, rho u, rho v, rho w, E), rows 5-9 w_x, rows 10-14 w_y,
 * rows 15-19 w_z.  Status codes and hfd_last_error() are those of hfd.h.  Every call that takes
 * a stream enqueues its kernels on it (NULL = the legacy default stream) and returns without
 * synchronising unless it says otherwise. */
#ifndef HFD3D_H
#define HFD3D_H

#include <stdint.h>

#include "hfd.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hfd3_mesh hfd3_mesh;

/* A periodic tetrahedral mesh of the box [0, Lx) x [0, Ly) x [0, Lz).  x, y, z: host arrays of
 * nv vertex coordinates; tet: host array of 4*ntet vertex ids.  Displacements between vertices
 * are taken by minimum image, so every edge must be shorter than half of each box length.  The
 * arrays are read during hfd3_mesh_create only (caller owned). */
typedef struct {
  int32_t nv;
  const double* x;
  const double* y;
  const double* z;
  int32_t ntet;
  const int32_t* tet;
  double Lx, Ly, Lz;
} hfd3_mesh_desc;

/* Parameters.  gamma: ratio of specific heats; weno_eps: epsilon of the WENO weights;
 * sens_lo, sens_hi: the sensor band of Eq. (2d_hweno_intp) (5-node value when
 * sens_lo < omega_1 < sens_hi); harten: Harten's entropy-fix width over c; sv_rtol: singular
 * values below sv_rtol * sigma_max of the 20 x 20 Hermite system count as zero before the
 * dropping rule; div_cond_min: a divergence stencil whose pivoted-QR estimate |R_nn| / |R_11|
 * falls below it makes hfd3_mesh_create fail with HFD_ERR_SINGULAR; force_branch: 0 sensor,
 * 1 every side 5-node, 2 every side weighted 3-node (testing aid); threads: host preprocessing
 * threads (0 = all hardware threads); host_only: 1 builds the host preprocessing only (no
 * device memory, no GPU needed: hfd3_prep_get and hfd3_mesh_info work, the device calls
 * return HFD_ERR_UNSUPPORTED), 0 also uploads it. */
typedef struct {
  double gamma, weno_eps, sens_lo, sens_hi, harten, sv_rtol, div_cond_min;
  int32_t force_branch;
  int32_t threads;
  int32_t host_only;
} hfd3_options;

/* gamma 1.4, weno_eps 1e-2, sens_lo 0.01, sens_hi 0.79, harten 0.1, sv_rtol 1e-13,
 * div_cond_min 1e-12, force_branch 0, threads 0, host_only 0. */
void hfd3_default_options(hfd3_options* opts);

/* Builds the mesh: host preprocessing in FP64 (edges sorted by (tail, head) with tail < head;
 * stencils, tangent frames, 5-node and 3-node weights per edge; divergence rows per vertex over
 * its two-level stencil) and upload of the device arrays.  opts NULL = defaults.  *out is
 * owned by the caller (hfd3_mesh_destroy).  Errors: HFD_ERR_ARG (null or inconsistent
 * description, an id out of range, a box length <= 0), HFD_ERR_SINGULAR (a stencil that cannot
 * be extended, a Hermite system with no singular value left, an ill-conditioned divergence
 * stencil), HFD_ERR_CUDA (allocation or copy). */
hfd_status hfd3_mesh_create(const hfd3_mesh_desc* desc, const hfd3_options* opts, hfd3_mesh** out);

void hfd3_mesh_destroy(hfd3_mesh* mesh);

/* info[0] vertices, info[1] edges, info[2] vertex entries and info[3] edge entries of the
 * divergence rows (sum over vertices of the stencil sizes), info[4] sides whose Hermite system
 * kept fewer than 20 singular values, info[5] host preprocessing time in microseconds. */
hfd_status hfd3_mesh_info(const hfd3_mesh* mesh, int64_t info[6]);

/* Host copies of the preprocessing, by name, with their element counts (E edges, V vertices,
 * Nv / Ne divergence entries):
 *   "edges" int32 2E (tail, head); "sten" int32 6E (the 6 stencil ids of each edge);
 *   "frame" float64 9E (n, t1, t2 of each edge); "w5" float64 40E (per edge, side L then R, the
 *   20 weights (v, x, y, z) per node); "w3" float64 18E (per edge, side, candidate: 3 weights);
 *   "rank" int32 2E; "vptr" int32 V+1 and "eptr" int32 V+1 (row pointers); "vidx" int32 Nv and
 *   "eidx" int32 Ne (vertex and edge ids); "cv" float64 12 Nv (per vertex entry, rows d_0, d_x,
 *   d_y, d_z times fluxes f, g, k); "ce" float64 4 Ne (per edge entry, the four rows).
 * hfd3_prep_size returns the count (-1 for an unknown name).  hfd3_prep_get copies count
 * elements to dst (host).  hfd3_prep_set overwrites "sten", "frame", "w5", "w3", "cv" or "ce"
 * from src (host, exactly the array's count) and uploads it again (synchronous); the
 * connectivity arrays are read-only.  Errors: HFD_ERR_ARG (unknown or read-only name, wrong
 * count, null pointer, a stencil id out of range), HFD_ERR_CUDA. */
int64_t hfd3_prep_size(const hfd3_mesh* mesh, const char* name);
hfd_status hfd3_prep_get(const hfd3_mesh* mesh, const char* name, void* dst, int64_t count);
hfd_status hfd3_prep_set(hfd3_mesh* mesh, const char* name, const void* src, int64_t count);

/* R = -div f(w), -div f_x, -div f_y, -div f_z (the 3D form of Eq. (HWENO)) for the state U.
 * U and R: 20*nv device arrays (distinct).  Three kernels: vertex fluxes, edge fluxes (Alg. 1
 * with Roe's flux), divergence gather.  Non-finite results set HFD_ERR_NONFINITE in the error
 * word (hfd3_check).  Errors: HFD_ERR_ARG, HFD_ERR_CUDA (launch). */
hfd_status hfd3_residual(hfd3_mesh* mesh, const double* U, double* R, void* stream);

/* nsteps SSP-RK3 steps (Sec. 2.3, end) of fixed size dt > 0, in place on U (20*nv device
 * array).  Each stage runs the vertex and edge kernels and the divergence kernel with the stage
 * update fused; the stages use the mesh's two scratch states.  A non-finite value or a
 * non-positive density sets HFD_ERR_NONFINITE / HFD_ERR_POSITIVITY in the error word.
 * Errors: HFD_ERR_ARG (dt <= 0, nsteps < 0, null pointer), HFD_ERR_CUDA. */
hfd_status hfd3_steps(hfd3_mesh* mesh, double* U, double dt, int32_t nsteps, void* stream);

/* hfd3_steps with every kernel bracketed by CUDA events: ms[0], ms[1], ms[2] receive the total
 * device time of the vertex, edge and divergence kernels over the nsteps steps.  Synchronises
 * the stream.  Errors: as hfd3_steps, and HFD_ERR_ARG for a null ms. */
hfd_status hfd3_steps_profiled(hfd3_mesh* mesh, double* U, double dt, int32_t nsteps, double ms[3],
                               void* stream);

/* Lanes (consecutive threads) per vertex in the divergence gather: 1, 2 or 4 (default 4).  The
 * lanes take the vertex's entries in turn and their sums are combined by a fixed butterfly, so
 * every count gives deterministic results that agree with the others to rounding.  Errors:
 * HFD_ERR_ARG (another count or a null mesh). */
hfd_status hfd3_mesh_set_lanes(hfd3_mesh* mesh, int32_t lanes);

/* Reads and clears the mesh's device error word (synchronises the device): HFD_OK, or the
 * first of HFD_ERR_MESH (a gathered index out of range, which the kernels skip),
 * HFD_ERR_NONFINITE, HFD_ERR_POSITIVITY recorded since the last check. */
hfd_status hfd3_check(hfd3_mesh* mesh);

#ifdef __cplusplus
}
#endif

#endif /* HFD3D_H */
