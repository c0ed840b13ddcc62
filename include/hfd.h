/*
 * hfd.h - C ABI of the GB300 Hermite finite-difference library.
 *
 * The library advances the semi-discrete system of the Hermite finite-difference method for
 * 2D Euler / Navier-Stokes on unstructured triangle meshes (Zhou, Zhen, Qu, Cai, arXiv
 * 2109.01286).  Each vertex carries 12 unknowns, w = (rho, rho u, rho v, E) and its
 * derivatives w_x, w_y (Eq. (HWENO), Sec. 2.3).  One right-hand-side evaluation is three
 * GPU kernels: analytic vertex fluxes (Sec. 2.3), Hermite-WENO interpolation plus a Riemann
 * flux at every edge midpoint (Alg. 1, Eq. (2d_hweno_intp)), and the two-level least-squares
 * divergence (Eq. (flux_polynomials) and the d_0/d_x/d_y rows), fused with the update of the
 * three-stage TVD Runge-Kutta scheme (Sec. 2.3, end).
 *
 * Conventions shared by every entry point:
 *  - Return value: HFD_OK or an hfd_status error code; no C++ exception crosses the ABI.  The
 *    message of the last error of the calling thread is hfd_last_error().
 *  - State arrays are 12 x V float64 structure-of-arrays (row r of vertex v at U[r*V + v]):
 *    rows 0-3 w, rows 4-7 w_x, rows 8-11 w_y.  Arrays passed to hfd_residual / hfd_step /
 *    hfd_steps are DEVICE pointers in the mesh's INTERNAL vertex order (space-filling-curve
 *    order, non-ghost vertices first).  hfd_state_import / hfd_state_export convert from / to
 *    the caller's input vertex order on the device.
 *  - Device calls are asynchronous on the given stream (0 = legacy default stream) unless the
 *    entry point says otherwise.  A mesh is not thread-safe: calls on one mesh must be
 *    serialised by the caller.  Distinct meshes are independent.
 *  - Pointers are caller-owned unless stated; the library copies what it keeps.
 */
#ifndef HFD_H
#define HFD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HFD_OK = 0,
  HFD_ERR_ARG = 1,         /* invalid argument (null pointer, size, option out of range)   */
  HFD_ERR_MESH = 2,        /* invalid mesh (bad triangle, index out of range, non-manifold) */
  HFD_ERR_STENCIL = 3,     /* an edge stencil cannot be assembled (Sec. 2.1)               */
  HFD_ERR_SINGULAR = 4,    /* a least-squares system has no usable singular value          */
  HFD_ERR_CUDA = 5,        /* CUDA runtime error (message carries cudaGetErrorString)      */
  HFD_ERR_NONFINITE = 6,   /* device error word: non-finite value produced                 */
  HFD_ERR_POSITIVITY = 7,  /* device error word: rho <= 0 or p <= 0 after an RK stage       */
  HFD_ERR_TIMEOUT = 8,     /* device error word: a bounded device wait gave up             */
  HFD_ERR_UNSUPPORTED = 9  /* option combination not built                                 */
} hfd_status;

/* Mesh description (Sec. 2.1 works on the edges of a triangulation).  Host pointers, copied. */
typedef struct {
  int32_t nv;              /* number of vertices (ghosts included)                          */
  int32_t ntri;            /* number of triangles                                           */
  const double* x;         /* nv vertex coordinates                                         */
  const double* y;
  const int32_t* tri;      /* 3*ntri vertex ids, counter-clockwise                          */
  double Lx, Ly;           /* domain extents; used for the minimum image on periodic axes   */
  int32_t periodic_x;      /* nonzero: displacements along x wrap with period Lx            */
  int32_t periodic_y;
  int32_t nghost;          /* transmissive ghost vertices (no residual, refreshed by copy)  */
  const int32_t* ghost_ids;    /* nghost ids                                                */
  const int32_t* ghost_donor;  /* nghost donor ids (non-ghost vertices), or -1: a fixed ghost
                                  (a wall band, Sec. 3.2) whose 12 values the caller sets in
                                  the state and no refresh changes                          */
  const int32_t* ghost_flags;  /* bit 0: zero w_x on refresh, bit 1: zero w_y               */
} hfd_mesh_desc;

/* Numerical options.  hfd_default_options fills the defaults shown. */
typedef struct {
  int32_t precision;       /* 0: FP64 throughout; 1: FP32 bulk (FP64 state, RK accumulation,
                              geometry solves, WENO weight ratios)                        [0] */
  int32_t div_degree;      /* degree of the LS divergence polynomials                     [5] */
  int32_t visc_degree;     /* degree of the viscous vertex-only LS                        [4] */
  int32_t viscous;         /* nonzero: add the viscous flux divergence                    [0] */
  int32_t renumber;        /* nonzero: internal order along a Hilbert curve               [1] */
  int32_t nthreads;        /* host preprocessing threads, 0 = all hardware threads        [0] */
  double gamma;            /* ratio of specific heats                                   [1.4] */
  double mu;               /* dynamic viscosity (constant)                                [0] */
  double prandtl;          /* Prandtl number                                           [0.72] */
  double R_gas;            /* gas constant, p = rho R T                                   [1] */
  double weno_eps;         /* epsilon of the WENO weights                              [1e-2] */
  double sens_lo;          /* smooth (5-node) branch iff sens_lo < omega_1 < sens_hi   [0.01] */
  double sens_hi;          /*                                                          [0.79] */
  double sv_rtol;          /* singular values <= sv_rtol*sigma_max count as zero      [1e-13] */
  double div_cond_min;     /* LS degree drops by one below this sigma ratio estimate  [1e-12] */
  double harten;           /* entropy-fix width as a fraction of the Roe sound speed    [0.1] */
  double cfl;              /* CFL number of the device time step                        [0.3] */
  double visc_coef_max;    /* viscous vertex-only LS: the degree drops by one (down to 2)
                              while a first- or second-derivative weight, in coordinates
                              scaled by the mean incident edge length, exceeds this       [8] */
  /* Device memory of a mesh (no counterpart in the paper).  NULL: cudaMalloc / cudaFree.
   * Otherwise every device block a mesh holds comes from dev_alloc(bytes, alloc_ctx) on the
   * current device and goes back through dev_free(ptr, alloc_ctx) in hfd_mesh_destroy, after a
   * device synchronisation (a caching allocator may hand the block out again at once).
   * dev_alloc must return memory aligned to 256 bytes, or NULL when it cannot; the library
   * then fails with HFD_ERR_CUDA.  Both or neither must be set (else HFD_ERR_ARG).
   * hfd_residual_static allocates nothing either way.                                 [NULL] */
  void* (*dev_alloc)(size_t bytes, void* alloc_ctx);
  void (*dev_free)(void* ptr, void* alloc_ctx);
  void* alloc_ctx;
  int32_t flux;            /* Riemann solver of the edge flux (Sec. 2.3 after Alg. 1; the paper
                              does not name one): 0 Roe with Harten's fix, 1 Rusanov       [0] */
  int32_t conservative;    /* 1: conservative variant, not in the paper (which names conservation
                              as open, Sec. 4): the value rows become the median-dual finite
                              volume divergence (1/|C_v|) sum_e +-|S_e| h_e, with S_e the
                              dual-face area vector of edge e, and every edge's projection and
                              Riemann flux is taken along S_e/|S_e|; the derivative rows stay
                              least squares (with edge rows along S_e)                    [0] */
  int32_t force_branch;    /* debugging and testing aid (Alg. 1's branch taken for every
                              characteristic component and side instead of the sensor's
                              choice): 0 the sensor decides, 1 the 5-node Hermite value,
                              2 the WENO-weighted 3-node candidates.  hfd_adjoint supports 0 [0] */
} hfd_options;

typedef struct {
  int64_t nv;              /* vertices                                                      */
  int64_t nactive;         /* non-ghost vertices (residual rows), internal ids [0, nactive) */
  int64_t nedges;          /* edges of the triangulation                                    */
  int64_t nflux_edges;     /* edges whose numerical flux some divergence row reads          */
  int64_t div_nnz;         /* total divergence row length (2N+M summed over active)         */
  int64_t div_nv_total;    /* total stencil vertices N summed over active vertices          */
  int64_t div_ne_total;    /* total stencil edges M summed over active vertices             */
  int32_t div_nv_max, div_ne_max;
  int64_t rank_hist[16];   /* 5-node ranks kept, over both sides of every flux edge         */
  int64_t div_degree_fallbacks;
  int64_t device_bytes;    /* device memory held by the mesh                                */
  double prep_seconds;     /* host preprocessing wall time                                  */
  int32_t nmember;         /* meshes in a batch (hfd_prep_concat), 1 otherwise              */
  int64_t visc_degree_fallbacks; /* viscous rows whose degree dropped (visc_coef_max)       */
} hfd_mesh_stats;

typedef struct hfd_prep hfd_prep;
typedef struct hfd_mesh hfd_mesh;

void hfd_default_options(hfd_options* opts);
const char* hfd_last_error(void);

/* ---------------------------------------------------------------- host preprocessing
 * hfd_prep_create runs the geometry-only preprocessing on the host in FP64 (no GPU needed):
 * edge list (Sec. 2.1), curvilinear 6-node stencils of every edge a divergence row reads
 * (Sec. 2.1, Fig. 1; extension by smallest deflection, ties to the lower input id), the
 * 5-node Hermite weights (first row of the pseudo-inverse of the 15x15 system of
 * Eq. (hintp_5), Sec. 2.2, with trial dropping of singular values), the 3-node weights of
 * Eq. (3nodes_intp), and the divergence rows d_0, d_x, d_y of Eq. (flux_polynomials) for every
 * non-ghost vertex (plus the viscous vertex-only rows if opts->viscous).
 * Errors: HFD_ERR_ARG, HFD_ERR_MESH, HFD_ERR_STENCIL, HFD_ERR_SINGULAR. */
hfd_status hfd_prep_create(const hfd_mesh_desc* desc, const hfd_options* opts, hfd_prep** out);
void hfd_prep_destroy(hfd_prep* prep);

/* Named arrays of a prep object, all in INPUT numbering.  hfd_prep_size returns the element
 * count of `name` (or -1); hfd_prep_get copies it out; hfd_prep_set overwrites it (same size;
 * only the coefficient arrays "w5", "w3", "div_coef", "visc_coef" are writable).  Names:
 *   "edges" int32 [E][2] (tail < head, sorted); "flux_edges" int32 [Ef] edge indices;
 *   "stencil" int32 [Ef][6]; "normal" f64 [Ef][2]; "w5" f64 [Ef][2][15] (side, node*3 +
 *   {value, x, y}); "w3" f64 [Ef][2][3][3] (side, sub-stencil, node); "rank" int32 [Ef][2];
 *   "active" int32 [A]; "div_vptr" int32 [A+1]; "div_vidx" int32; "div_eptr" int32 [A+1];
 *   "div_eidx" int32 (edge indices); "div_coef" f64, per active vertex a block of
 *   3 x (2N+M) (rows d_0, d_x, d_y over the data [f_1, g_1, ..., f_N, g_N, h_1..h_M]);
 *   "div_degree" int32 [A]; "visc_coef" f64, per active vertex 3 x 2N. */
int64_t hfd_prep_size(const hfd_prep* prep, const char* name);
hfd_status hfd_prep_get(const hfd_prep* prep, const char* name, void* dst, int64_t count);
hfd_status hfd_prep_set(hfd_prep* prep, const char* name, const void* src, int64_t count);

/* Batches (many independent meshes advanced together): the disjoint union of n prep objects
 * with identical physical and numerical options.  Member k's vertices (edges) follow those of
 * members 0..k-1 in the input numbering of the result, so a batch state is the concatenation
 * of the members' states.  The device mesh made from it runs every kernel once over all members
 * and gives each member its own CFL time step (hfd_step with dt <= 0); hfd_last_dt then returns
 * n values.  The inputs are not consumed.  Errors: HFD_ERR_ARG. */
hfd_status hfd_prep_concat(const hfd_prep* const* preps, int32_t n, hfd_prep** out);

/* ---------------------------------------------------------------- batches, one array per member
 * The batch form of Sec. 3's test problems, with one state array per member mesh (the
 * concatenated form is hfd_prep_concat + hfd_mesh_upload, whose single state holds all members).
 * hfd_batch_create: the disjoint union of n preps uploaded in `precision` (-1 / 0 / 1 as in
 * hfd_mesh_upload).  hfd_batch_step advances every member by one SSP-RK3 step (Sec. 2.3, end)
 * in one pass of the kernels: U[k] is member k's 12 x nv_k device state in its own input order
 * (updated in place); dt is n positive steps (host array), or NULL for each member's own CFL
 * step.  It gathers the members into the batch's array, steps it, scatters the result back,
 * and returns after the stream has finished (the host arrays U and dt may then be reused).
 * hfd_batch_mesh lends the union mesh (owned by the batch) for the other hfd_mesh calls, e.g.
 * hfd_last_dt.  Errors: HFD_ERR_ARG, HFD_ERR_CUDA, and those of hfd_prep_concat and
 * hfd_mesh_upload. */
typedef struct hfd_batch hfd_batch;
hfd_status hfd_batch_create(const hfd_prep* const* preps, int32_t n, int32_t precision,
                            hfd_batch** out);
void hfd_batch_destroy(hfd_batch* batch);
hfd_status hfd_batch_mesh(hfd_batch* batch, hfd_mesh** mesh);
hfd_status hfd_batch_step(hfd_batch* batch, double* const* U, const double* dt, void* stream);

/* ---------------------------------------------------------------- device mesh
 * hfd_mesh_create = hfd_prep_create + hfd_mesh_upload.  hfd_mesh_upload renumbers vertices
 * and edges (Hilbert order of coordinates; non-ghost vertices first) and uploads the
 * structure-of-arrays coefficient streams in the requested precision to the current device.
 * The prep object is not consumed.  Errors: as hfd_prep_create, HFD_ERR_CUDA. */
hfd_status hfd_mesh_create(const hfd_mesh_desc* desc, const hfd_options* opts, hfd_mesh** out);
/* precision: -1 = the prep's option, 0 = FP64, 1 = FP32 bulk (one prep can feed both). */
hfd_status hfd_mesh_upload(const hfd_prep* prep, int32_t precision, hfd_mesh** out);
void hfd_mesh_destroy(hfd_mesh* mesh);
hfd_status hfd_mesh_info(const hfd_mesh* mesh, hfd_mesh_stats* out);
/* perm[internal id] = input vertex id (host array of nv entries). */
hfd_status hfd_mesh_perm(const hfd_mesh* mesh, int32_t* perm);

/* Device permutation of 12 x V state arrays between input order and internal order. */
hfd_status hfd_state_import(hfd_mesh* mesh, const double* U_input, double* U_internal,
                            void* stream);
hfd_status hfd_state_export(hfd_mesh* mesh, const double* U_internal, double* U_input,
                            void* stream);

/* Right-hand side R(U) of Eq. (HWENO): rows 0-3 -div f, rows 4-7 -div f_x, rows 8-11 -div f_y
 * (plus the viscous divergences), zero at ghost vertices.  The ghost columns of U are refreshed
 * in place first (transmissive copy from the donor, flagged derivatives zeroed).  U and R are
 * 12*nv device arrays in internal order and must not overlap. */
hfd_status hfd_residual(hfd_mesh* mesh, double* U, double* R, void* stream);

/* One step of the three-stage TVD Runge-Kutta scheme (Sec. 2.3), in place on U:
 * u1 = u + dt R(u); u2 = 3/4 u + 1/4 (u1 + dt R(u1)); u <- 1/3 u + 2/3 (u2 + dt R(u2)).
 * Only non-ghost vertices advance; ghost columns are refreshed at the end.  dt > 0 is used as
 * given; dt <= 0 selects dt = cfl * min_v l_min(v) / (|u| + c) computed on the device from
 * the step's initial state (no host synchronisation). */
hfd_status hfd_step(hfd_mesh* mesh, double* U, double dt, void* stream);

/* nsteps calls of hfd_step, replayed from a CUDA graph captured on the first call for this
 * (U, dt mode).  Same semantics as nsteps calls of hfd_step. */
hfd_status hfd_steps(hfd_mesh* mesh, double* U, double dt, int32_t nsteps, void* stream);

/* End-to-end form with HOST buffers in input order: copies U_in (12*nv doubles, ideally
 * pinned) to the device, imports it, runs nsteps steps, exports and copies the result to
 * U_out (may equal U_in), then synchronises the stream.  Uses mesh-owned device buffers. */
hfd_status hfd_steps_host(hfd_mesh* mesh, const double* U_in, double* U_out, double dt,
                          int32_t nsteps, void* stream);

/* Same work as hfd_steps, launched kernel by kernel with CUDA events recorded around each
 * launch on `stream`; synchronises the stream and accumulates into kernel_ms[6] the time spent
 * in each kernel kind: [0] ghost refresh, [1] vertex fluxes, [2] edge interpolation + Riemann
 * flux, [3] divergence + RK stage, [4] time-step reduction, [5] persistent stage kernel.
 * Returns in *launches the number of kernels launched (the time-step reduction is two).
 * Tracing aid: events add a few microseconds each. */
hfd_status hfd_steps_profiled(hfd_mesh* mesh, double* U, double dt, int32_t nsteps, void* stream,
                              double* kernel_ms, int64_t* launches);

/* hfd_residual without device allocation.  The paper has no counterpart: this entry point is
 * for callers that cannot allocate device memory when they evaluate residuals -- applications
 * that reserve all device memory for their own pool up front, and code that must not call
 * cudaMalloc/cudaFree (which can synchronise the device) while other work runs.  Same inputs,
 * output and result as hfd_residual (U in/out for its ghost columns, R out, both 12*nv device
 * arrays in internal order), but the per-call scratch (state copy, vertex and edge fluxes) is a
 * fixed 8 MiB array compiled into the library, held on every GPU that loads the library until
 * the process exits.  That is room for about 32,000 vertices in FP64 (256 bytes each with their
 * ~3 flux edges) or 65,000 in FP32 bulk; larger meshes get HFD_ERR_ARG with the bytes needed.
 * Every call looks up the array's device address (cudaGetSymbolAddress, with the mesh's device
 * current), so the address stays right across a cudaDeviceReset; the first call on a device
 * may also load the library's device code there, so make that first call before any stream
 * capture.  All calls on a
 * device share the array: calls that overlap on the GPU race and must be serialised by the
 * caller.  Every call rewrites what it reads, so nothing carries over between calls.  Errors:
 * HFD_ERR_ARG (sizes, null pointers, mesh not on the current device), HFD_ERR_CUDA. */
hfd_status hfd_residual_static(hfd_mesh* mesh, double* U, double* R, void* stream);

/* Measured fused multiply-add throughput of the current device, for the arithmetic roofline of
 * the FP64 path.  The paper has no counterpart: this is a measurement aid.  Hand-written loops
 * of independent FMA chains (no memory traffic) run on every SM for about 25 ms per launch, in
 * FP64 and then FP32; the best of three timed launches (after one warm-up) is returned as
 * FLOP/s (2 per FMA) in *fp64_flops and *fp32_flops, and the device's SM count
 * (cudaDevAttrMultiProcessorCount) in *sm_count.  The figures are at the clocks the device
 * runs during the call.  Allocates and frees a small device buffer; synchronises the stream.
 * Errors: HFD_ERR_ARG (null output), HFD_ERR_CUDA. */
hfd_status hfd_measure_fma_peaks(double* fp64_flops, double* fp32_flops, int32_t* sm_count,
                                 void* stream);

/* Discrete adjoint of one step (gradients through the time stepping): given
 * lam_np1 = dJ/dU_{n+1}, writes lam_n = (d hfd_step(U_n, dt) / d U_n)^T lam_np1, the exact
 * vector-Jacobian product of the discrete step (Sec. 2.3: Alg. 1, Riemann flux, least-squares
 * divergence, three-stage TVD Runge-Kutta) with the branch decisions of the sensor held fixed.
 * The three stages are recomputed forward from U_n (not modified), then reversed; the
 * divergence and stencil transposes are gathers over lists built on the first call, so the
 * result is deterministic.  All arrays are 12*nv device arrays in internal order; dt > 0 is the
 * fixed step of the forward step (a step with dt <= 0 depends on U_n through the CFL minimum,
 * which this product does not differentiate).  Ghost layers enter transposed: a transmissive
 * ghost's sensitivity goes to its donor (without the derivative rows the refresh zeroes) and
 * its column of lam_n is zero; a fixed ghost (donor -1) is an input of every stage, and its
 * column of lam_n holds that sensitivity.  Viscous meshes add the reverse of the vertex
 * viscous fluxes and the transposed viscous rows.  Roe or Rusanov flux.  A batch
 * (hfd_prep_concat) takes the one dt for every member, and its product is each member's.
 * FP64 meshes; FP32 meshes get HFD_ERR_UNSUPPORTED.  Errors: HFD_ERR_ARG, HFD_ERR_CUDA. */
hfd_status hfd_adjoint(hfd_mesh* mesh, const double* U_n, const double* lam_np1, double* lam_n,
                       double dt, void* stream);

/* How hfd_step runs a Runge-Kutta stage.  persistent = 0: four launches (ghost refresh, vertex
 * fluxes, edge fluxes, divergence + stage update).  persistent = 1: one cooperative launch of
 * `grid` blocks (0 = every co-resident block) running the same four phases separated by
 * bounded grid barriers (a wait that exceeds its bound records HFD_ERR_TIMEOUT, see hfd_check).
 * Both run the same per-entity code; they agree to rounding (the compiler may contract
 * multiply-adds differently in the fused kernel).  Drops captured graphs.  Errors: HFD_ERR_ARG. */
hfd_status hfd_mesh_set_launch(hfd_mesh* mesh, int32_t persistent, int32_t grid);

/* Bound on the polls of one grid-barrier wait in the persistent launch (default 2^24 polls of
 * at least 64 ns).  A smaller bound makes a stalled wait give up sooner: the kernel then records
 * HFD_ERR_TIMEOUT in the error word and returns instead of waiting.  Drops captured graphs. */
hfd_status hfd_mesh_set_barrier_limit(hfd_mesh* mesh, uint32_t polls);

/* Lanes (threads) per vertex in the divergence gather: 1, 2, 4 or 8.  The defaults are 1 for
 * FP64 meshes (FP64-pipe bound: no cross-lane reduction) and 4 for FP32 meshes (memory bound:
 * coalesced groups); small meshes fill the GPU better with more lanes.  Each lane sums a
 * strided share of the entries and the shares are combined by a fixed reduce-scatter, so a lane
 * count gives deterministic results that agree with the other counts to rounding.  The
 * persistent form (hfd_mesh_set_launch) has kernels for 1, 2 and 4 lanes and runs 8 as 4.  Drops
 * captured graphs.  Errors: HFD_ERR_ARG (another count, or a persistent grid set by
 * hfd_mesh_set_launch that the new count's kernel cannot hold co-resident). */
hfd_status hfd_mesh_set_lanes(hfd_mesh* mesh, int32_t lanes);

/* Testing aid: the branch of Alg. 1 (Eq. (2d_hweno_intp)) that the edge kernel takes on state U
 * (12*nv device array, internal order; its ghost columns are refreshed): runs the ghost refresh,
 * vertex fluxes and edge kernel once and writes, for every flux edge in the preprocessing's
 * flux-edge order ("flux_edges" of hfd_prep_get), one byte to the HOST array branches[nflux_edges]
 * (caller owned): bit side*4+q is set where characteristic component q of side L (0) or R (1)
 * took the WENO-weighted 3-node value instead of the 5-node one.  The decision is the path's
 * own (FP32 sensor with FP64 re-decision inside a guard band on FP64 meshes).  Allocates a
 * temporary device block; synchronises the stream.  Errors: HFD_ERR_ARG, HFD_ERR_CUDA. */
hfd_status hfd_edge_branches(hfd_mesh* mesh, double* U, uint8_t* branches, void* stream);

/* Testing aid: the integer-only FP64/FP32 conversions of the kernels beside the hardware
 * conversions.  The FP64 kernels round their FP32 sensor inputs, and the FP32 kernels widen
 * their sums for the FP64 stage update, with integer operations: GB300 converts between FP64
 * and FP32 at its FP64 rate.  For each of the n doubles x[i] (device array) writes
 * f_int[i] = x[i] rounded to float by the integer form, f_hw[i] = the hardware's round to
 * nearest, and, for the float whose bits are the low 32 bits of x[i], d_int[i] = that float
 * widened by the integer form, d_hw[i] = the hardware widening (device arrays of n, caller
 * owned).  The two of each pair are equal bit for bit except on NaN (both NaN).  Errors:
 * HFD_ERR_ARG (n < 0 or a null array with n > 0), HFD_ERR_CUDA. */
hfd_status hfd_check_conversions(int64_t n, const double* x, float* f_int, float* f_hw,
                                 double* d_int, double* d_hw, void* stream);

/* Arithmetic of the FP64 divergence (the default is 0).  folded = 1: each least-squares row
 * (Eq. (flux_polynomials), the d_0, d_x, d_y rows) is evaluated as
 *   sum_j a'_j (F_j - F_c) + F_c sum_j a'_j + sum_m d_m dh_m,
 * where F_c is the row's own vertex flux, a' the vertex coefficients with each edge row's
 * endpoint average (1/2) d_m (F_a + F_b) . n_m folded in (at upload), and dh_m the edge flux
 * minus that average (written by the edge kernel).  The rows annihilate constant fluxes, so the
 * remaining terms are small, and the products run in double-float (pairs of FP32 values,
 * 48-bit significands) on the FP32 pipe; the differences, row sums and final combination stay
 * FP64.  Accuracy: equal to the plain evaluation within 1e-12 relative on the vortex, the
 * four-quadrant problem and the circular Sod mesh; on low-Mach flows the energy flux's nearly
 * divergence-free part still cancels (at Mach 0.1, about 250x), and the 48-bit products leave
 * ~1e-11 relative there, against ~1e-12 for the plain form.  Speed on the four-quadrant
 * 1024x1024 mesh (GB300): the divergence 1.66 ms against 2.23 ms, the edge kernel 0.11 ms
 * slower (it forms dh), the step 11.05 ms against 12.45 ms.  The viscous rows stay FP64.
 * folded = 0: the plain form, 24 FP64 multiply-adds per stencil vertex and 12 per stencil edge
 * on the FP64 pipe, with the lane count of hfd_mesh_set_lanes.  Drops captured graphs.
 * Errors: HFD_ERR_ARG (folded not 0 or 1), HFD_ERR_UNSUPPORTED (folded = 1 on an FP32 mesh). */
hfd_status hfd_mesh_set_fp64_div(hfd_mesh* mesh, int32_t folded);

/* Divergence kernel of an FP32-bulk mesh (the default is 0).  staged = 1: the staged kernel --
 * a persistent, warp-specialised grid walks tiles of consecutive vertices whose row pointers,
 * index chunks and coefficient chunks (the contiguous streams of the least-squares rows, Eq.
 * (flux_polynomials)) one producer thread copies into shared memory with 1D bulk copies, up to
 * three tiles ahead of eight consumer warps; 8 lanes per vertex.  staged = 0: the unstaged
 * kernel with the lane count of hfd_mesh_set_lanes, which holds more vertices' gathers in
 * flight per SM and measured faster on the four-quadrant 1024x1024 mesh (0.395 ms against
 * 0.560 ms per launch on a GB300); the autotuner times both.  The two agree to rounding (bit
 * for bit at 8 lanes).  staged = 2 (inviscid FP32-bulk meshes): the gather-staged kernel --
 * each block of 256 threads takes 64 consecutive vertices at 4 lanes each, first copies the
 * vertex fluxes and edge fluxes that their rows read, each distinct one once, into shared
 * memory (lists built at upload, with every chunk's indices rewritten as 16-bit positions in
 * them), then runs the unstaged kernel's chunk loop against shared memory; bit for bit equal to
 * the unstaged kernel at 4 lanes, and measured slower on the four-quadrant 1024x1024 mesh
 * (0.433 ms against 0.395 ms per launch: the unstaged kernel's gathers already hit L1/L2, its
 * limit is the coefficient stream, and the staging pass adds a round of loads and a barrier
 * before any arithmetic).  Drops captured graphs.  Errors: HFD_ERR_ARG (staged not 0,
 * 1 or 2), HFD_ERR_UNSUPPORTED (staged = 1 on an FP64 mesh, staged = 2 on an FP64 or viscous
 * mesh or one whose tile lists would exceed 160 KB of shared memory). */
hfd_status hfd_mesh_set_div_staged(hfd_mesh* mesh, int32_t staged);

/* Autotuner: times one Runge-Kutta stage on (a copy of) the device state U, internal order,
 * for every lane count of hfd_mesh_set_lanes in the four-launch form (unstaged divergence),
 * for the staged divergence of an FP32-bulk mesh (hfd_mesh_set_div_staged), and for 1, 2 and 4
 * lanes in the persistent form at every co-resident block count; keeps the fastest, and writes
 * it to choice[0] (persistent), choice[1] (grid), choice[2] (lanes) and choice[3] (staged) if
 * choice (4 int32, caller owned) is not NULL.  The choice changes the launch shape and the
 * divergence's summation order, not the method's arithmetic (results agree to rounding, see
 * hfd_mesh_set_launch and hfd_mesh_set_lanes).  Synchronises. */
hfd_status hfd_mesh_autotune(hfd_mesh* mesh, const double* U, void* stream, int32_t* choice);

/* dt used by the most recent step, one value per member mesh (synchronises the stream). */
hfd_status hfd_last_dt(hfd_mesh* mesh, double* dt, void* stream);

/* Reads and clears the device error word (synchronises the stream): HFD_OK if clean, else the
 * first recorded error (HFD_ERR_NONFINITE, HFD_ERR_POSITIVITY). */
hfd_status hfd_check(hfd_mesh* mesh, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* HFD_H */
